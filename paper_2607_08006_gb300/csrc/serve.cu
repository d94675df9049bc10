// Serving: a persistent, device-resident progress kernel draining a host request ring
// with memory-based admission and tile-level continuous batching, and the plain
// launch-per-request path it is compared with.  (Persistent kernels and their progress:
// paper Sec. 3 and 7; the operations are the RMA, AMO and collectives of Sec. 6.3.)
//
// Roles in the server kernel:
//  * CTA 0, thread 0 -- the admitter: acquire-polls the ring tail in mapped host memory,
//    validates the request, finds a free slot and its destination pages (one page range
//    free on every PE the request writes: OR of the per-PE page bitmaps, first fit), marks
//    them, fills the slot and publishes (slot, generation) to the device work queue.
//  * CTAs 1..W -- workers: take tiles of queued requests (a window of the queue's oldest
//    entries, spread by CTA index so small requests run beside big ones), claim a tile by
//    compare-and-swap on the slot's (generation, next tile) word, run it, add its output
//    checksum, and count it done.  The CTA that completes the last tile writes the
//    completion record to mapped host memory, frees the pages and releases the slot.
// Every wait is bounded: the kernel exits on the stop flag once drained, after idle_ns
// without work, or after max_ns.
#include <cuda_runtime.h>
#include <time.h>

#include <cstring>
#include <thread>

#include "internal.h"
#include "quant_dev.cuh"

namespace shmemg {

constexpr int SV_THREADS = 256;   // CTAs of the plain path and of the server (two per SM)
constexpr int SRV_THREADS = SV_THREADS;
constexpr uint64_t RMA_TILE = 64ull << 10;    // bytes per put/get tile
constexpr uint64_t RED_TILE = 8192;           // elements per reduce tile
constexpr uint64_t A2A_TILE = 32ull << 10;    // bytes per alltoall block chunk
constexpr uint32_t WINDOW = 32;               // queue entries workers spread over
constexpr uint8_t FMT_F32 = 0xFF;

struct SvHost {                      // mapped host memory
    volatile uint64_t tail;          // requests published by the host
    uint8_t p0[120];
    volatile uint64_t head;          // requests taken by the admitter
    uint8_t p1[120];
    volatile uint32_t stop;
    uint8_t p2[124];
    volatile uint64_t consumed;      // completion records read by the host
    uint8_t p3[120];
};

constexpr uint32_t SV_MAX_SMID = 1024;
constexpr uint64_t SECONDARY_DELAY_NS = 1000;  // head start of each SM's first worker on a new request

struct SvCtl {                       // device memory
    unsigned long long fifo_head;
    uint8_t p0[120];
    unsigned long long fifo_tail;
    uint8_t p1[120];
    unsigned int exit_flag;
    uint8_t p2[124];
    unsigned long long comp_pos;
    uint8_t p3[120];
    unsigned long long inflight;
    uint8_t p4[120];
    unsigned long long consumed_cache;  // last host `consumed` value seen by the device
    uint8_t p5[120];
    unsigned int sm_workers[SV_MAX_SMID];  // worker CTAs per SM id (each worker's rank on its SM)
};

// One admitted request.  The claim word, which every worker that looks at the request
// touches, has a cache line of its own; the completion count and checksum (one update
// per published chunk) share another; the request fields are read-mostly.
struct __align__(128) SvSlot {
    shmemg_req_t req;
    uint64_t dst_off;
    uint32_t page0, npages;
    uint32_t ntiles, gen;
    uint64_t t_admit;
    uint64_t t_pub;                  // when the admitter queued it
    int32_t status;
    unsigned int busy;
    uint32_t nstage;                 // staging tiles (the first ones) of a staged request
    uint8_t pad0[128 - 116];
    unsigned long long claim;        // (gen << 32) | next tile
    uint8_t pad1[120];
    unsigned int done;
    unsigned int staged;             // finished staging tiles (release adds; op tiles acquire)
    unsigned long long checksum;
    uint8_t pad3[112];
};
static_assert(sizeof(SvSlot) == 384, "slot layout");

struct SvArgs {
    uint8_t *heap;
    uint64_t H;
    int npes;
    shmemg_server_cfg_t cfg;
    uint32_t pages_per_pe, bm_words;
    unsigned long long *bitmaps;     // npes * bm_words
    SvSlot *slots;
    uint32_t nslots;
    unsigned long long *fifo;        // (gen << 32) | slot
    uint32_t fifo_cap;
    SvCtl *ctl;
    SvHost *host;
    shmemg_req_t *ring;
    shmemg_completion_t *comp;
    uint32_t ring_slots;
};

__device__ __forceinline__ uint64_t now_dev() { return shmemg_d_globaltimer(); }

// ------------------------------------------------------------------ request geometry
struct Geo {
    int first, count;       // PEs (a contiguous range) whose pages the request takes
    int first2, count2;     // a second PE (staged put/get: the source PE), count2 = 0 if none
    uint64_t bytes;         // bytes per such PE: the destination, or a staged request's region
    uint32_t ntiles;        // all tiles: staging tiles first, then the operation's
    uint32_t nstage;        // staging tiles (0 unless the request stages its payload)
    int valid;
};

__host__ __device__ inline uint64_t round16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

// Offsets, from the region's start, of a staged request's source part (and of a bf16
// reduction's scales), per the layout of shmemg_req_t's staged payloads.
struct StagedParts {
    uint64_t src, scales;
};
__host__ __device__ inline StagedParts staged_parts(const shmemg_req_t &r) {
    StagedParts p = {0, 0};
    if (r.kind == SHMEMG_OP_PUT || r.kind == SHMEMG_OP_GET) {
        p.src = round16(r.n);
    } else if (r.kind == SHMEMG_OP_REDUCE) {
        if (r.dtype == SHMEMG_FLOAT && r.fmt == SHMEMG_FMT_BF16) {
            p.src = round16(4 * r.n);
            p.scales = p.src + round16(2 * r.n);
        }
    } else if (r.kind == SHMEMG_OP_ALLTOALL) {
        p.src = (uint64_t)r.issuer * r.n;
    }
    return p;
}

__host__ __device__ inline Geo geometry(const shmemg_req_t &r, int npes, uint64_t H, uint64_t amo_words) {
    Geo g = {0, 0, 0, 0, 0, 0, 0, 0};
    const bool staged = (r.flags & SHMEMG_REQ_STAGED) != 0;
    if (r.flags & ~(uint16_t)SHMEMG_REQ_STAGED) return g;
    switch (r.kind) {
    case SHMEMG_OP_PUT:
    case SHMEMG_OP_GET: {
        const int w = r.kind == SHMEMG_OP_PUT ? r.pe : r.issuer, sp = r.kind == SHMEMG_OP_PUT ? r.issuer : r.pe;
        if (r.pe < 0 || r.pe >= npes || r.issuer < 0 || r.issuer >= npes || r.n == 0 || (r.n & 7) || r.n > H)
            return g;
        if (!staged && ((r.src & 15) || r.src > H || r.n > H - r.src)) return g;
        g.first = w;
        g.count = 1;
        g.ntiles = (uint32_t)((r.n + RMA_TILE - 1) / RMA_TILE);
        if (staged) {
            g.bytes = 2 * round16(r.n);
            if (sp != w) {
                g.first2 = sp;
                g.count2 = 1;
            }
            g.nstage = g.ntiles;
            g.ntiles *= 2;
        } else {
            g.bytes = r.n;
        }
        break;
    }
    case SHMEMG_OP_FETCH_ADD:
    case SHMEMG_OP_COMPARE_SWAP:
    case SHMEMG_OP_FETCH_XOR:
        if (staged || r.dtype != SHMEMG_INT64 || amo_words == 0 || r.word >= (uint64_t)npes * amo_words) return g;
        g.ntiles = 1;
        break;
    case SHMEMG_OP_REDUCE: {
        int P = r.issuer;
        uint64_t in_es, out_es;
        if (r.dtype == SHMEMG_INT64) { in_es = 8; out_es = 8; }
        else if (r.dtype == SHMEMG_FLOAT && r.fmt == FMT_F32) { in_es = 4; out_es = 4; }
        else if (r.dtype == SHMEMG_FLOAT && r.fmt == SHMEMG_FMT_BF16) { in_es = 2; out_es = 4; }
        else return g;
        if (P < 1 || r.pe < 0 || (int64_t)r.pe + P > npes || r.n == 0 || (r.n & 3) || r.n > H) return g;
        const bool bf = r.fmt == SHMEMG_FMT_BF16 && r.dtype == SHMEMG_FLOAT;
        if (!staged) {
            if ((r.src & 15) || r.src > H || r.n * in_es > H - r.src) return g;
            if (bf) {
                uint64_t sb = (r.n + 127) / 128 * 4;
                if (r.cond < 0 || ((uint64_t)r.cond & 3) || (uint64_t)r.cond > H || sb > H - (uint64_t)r.cond) return g;
            }
        }
        g.first = r.pe;
        g.count = P;
        g.ntiles = (uint32_t)((r.n + RED_TILE - 1) / RED_TILE);
        if (staged) {
            const StagedParts sp = staged_parts(r);
            g.bytes = bf ? sp.scales + round16((r.n + 127) / 128 * 4) : r.n * out_es;  // fp32, int64: in place
            g.nstage = g.ntiles;
            g.ntiles *= 2;
        } else {
            g.bytes = r.n * out_es;
        }
        break;
    }
    case SHMEMG_OP_ALLTOALL: {
        int P = r.issuer;
        if (P < 1 || r.pe < 0 || (int64_t)r.pe + P > npes || r.n == 0 || (r.n & 15) || r.n > H ||
            r.n * (uint64_t)P > H)
            return g;
        if (!staged && ((r.src & 15) || r.src > H || r.n * (uint64_t)P > H - r.src)) return g;
        const uint64_t nt = (uint64_t)P * P * ((r.n + A2A_TILE - 1) / A2A_TILE);
        if (nt > (1u << 29)) return g;  // tile indices stay far inside 32 bits
        g.first = r.pe;
        g.count = P;
        g.ntiles = (uint32_t)nt;
        if (staged) {
            g.bytes = 2 * r.n * (uint64_t)P;
            g.nstage = (uint32_t)((uint64_t)P * ((r.n * (uint64_t)P + A2A_TILE - 1) / A2A_TILE));
            g.ntiles += g.nstage;
        } else {
            g.bytes = r.n * (uint64_t)P;
        }
        break;
    }
    default:
        return g;
    }
    g.valid = 1;
    return g;
}

// PE of member m of the request's page set (the first range, then the second)
__host__ __device__ inline int geo_pe(const Geo &g, int m) { return m < g.count ? g.first + m : g.first2 + (m - g.count); }

// ------------------------------------------------------------------ tiles
__device__ __forceinline__ uint64_t ck4(uint4 x, uint64_t i) {
    return (uint64_t)x.x * (2 * i + 1) + (uint64_t)x.y * (2 * i + 3) + (uint64_t)x.z * (2 * i + 5) +
           (uint64_t)x.w * (2 * i + 7);
}
__device__ __forceinline__ uint64_t ck2(uint2 x, uint64_t i) {
    return (uint64_t)x.x * (2 * i + 1) + (uint64_t)x.y * (2 * i + 3);
}

// bytes [b0, b1) of src -> dst; returns this thread's checksum terms, word index of
// byte b of the output = wbase + b / 4
__device__ __forceinline__ uint64_t copy_ck(uint8_t *dst, const uint8_t *src, uint64_t b0, uint64_t b1, uint64_t wbase) {
    uint64_t acc = 0;
    if (((uint64_t)dst | (uint64_t)src | b0 | b1) % 16 == 0) {
        const uint4 *s = (const uint4 *)src;
        uint4 *d = (uint4 *)dst;
        uint64_t v = b0 / 16 + threadIdx.x;
        const uint64_t e = b1 / 16, st = blockDim.x;
        for (; v + 7 * st < e; v += 8 * st) {  // eight 16-byte loads in flight per thread
            uint4 x[8];
#pragma unroll
            for (int u = 0; u < 8; u++) x[u] = __ldcg(s + v + u * st);
#pragma unroll
            for (int u = 0; u < 8; u++) {
                d[v + u * st] = x[u];
                acc += ck4(x[u], wbase + 4 * (v + u * st));
            }
        }
        for (; v + 3 * st < e; v += 4 * st) {
            uint4 a = __ldcg(s + v), b = __ldcg(s + v + st), c = __ldcg(s + v + 2 * st), f = __ldcg(s + v + 3 * st);
            d[v] = a;
            d[v + st] = b;
            d[v + 2 * st] = c;
            d[v + 3 * st] = f;
            acc += ck4(a, wbase + 4 * v) + ck4(b, wbase + 4 * (v + st)) + ck4(c, wbase + 4 * (v + 2 * st)) +
                   ck4(f, wbase + 4 * (v + 3 * st));
        }
        for (; v < e; v += st) {
            uint4 a = __ldcg(s + v);
            d[v] = a;
            acc += ck4(a, wbase + 4 * v);
        }
    } else {
        const uint2 *s = (const uint2 *)src;
        uint2 *d = (uint2 *)dst;
        for (uint64_t v = b0 / 8 + threadIdx.x; v < b1 / 8; v += blockDim.x) {
            uint2 a = __ldcg(s + v);
            d[v] = a;
            acc += ck2(a, wbase + 2 * v);
        }
    }
    return acc;
}

// ------------------------------------------------------------------ staged payloads
// Staged payload words (shmemg_req_t's definition): word q (0..3) of the counter draw z
// holds bytes 7 - 2q and 6 - 2q of z as two bfloat16 codes b(k) = sign of k's top bit,
// exponent 127, mantissa k's low 7 bits -- (-1)^(k >> 7) * (1 + (k & 127) / 128) --
// built with integer operations on both halves at once.
__device__ __forceinline__ uint32_t payload_of(uint64_t z, uint32_t q) {
    const uint32_t t = (uint32_t)(z >> (48 - 16 * q)) & 0xFFFFu;  // the word's two bytes
    const uint32_t u = ((t & 0xFF00u) << 8) | (t & 0xFFu);        // one per half-word
    return ((u & 0x00800080u) << 8) | 0x3F803F80u | (u & 0x007F007Fu);
}
__device__ __forceinline__ uint32_t payload_word(uint64_t seed, int p, uint64_t j) {
    return payload_of(cb64(seed, ((uint64_t)p << 40) | (j >> 2)), (uint32_t)(j & 3));
}
// words [j0, j1) of PE p's source part, which starts at `part` (16-byte aligned): four
// words -- one draw -- per 16-byte store where the range allows, single words at its ends
__device__ void stage_words(uint8_t *part, uint64_t seed, int p, uint64_t j0, uint64_t j1) {
    uint32_t *w = (uint32_t *)part;
    const uint64_t a0 = (j0 + 3) & ~(uint64_t)3, a1 = j1 & ~(uint64_t)3;
    if (a0 >= a1) {
        for (uint64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) w[j] = payload_word(seed, p, j);
        return;
    }
    for (uint64_t j = j0 + threadIdx.x; j < a0; j += blockDim.x) w[j] = payload_word(seed, p, j);
    // four independent draws per thread and pass: a draw is one serial chain of 64-bit
    // multiplies, so one chain per thread leaves the schedulers waiting on its latency
    const uint64_t nq = a1 / 4, bd = blockDim.x, hi = (uint64_t)p << 40;
    uint64_t q = a0 / 4 + threadIdx.x;
    for (; q + 3 * bd < nq; q += 4 * bd) {
        uint64_t z[4];
#pragma unroll
        for (int u = 0; u < 4; u++) z[u] = cb64(seed, hi | (q + u * bd));
#pragma unroll
        for (int u = 0; u < 4; u++)
            ((uint4 *)part)[q + u * bd] =
                make_uint4(payload_of(z[u], 0), payload_of(z[u], 1), payload_of(z[u], 2), payload_of(z[u], 3));
    }
    for (; q < nq; q += bd) {
        const uint64_t z = cb64(seed, hi | q);
        ((uint4 *)part)[q] = make_uint4(payload_of(z, 0), payload_of(z, 1), payload_of(z, 2), payload_of(z, 3));
    }
    for (uint64_t j = a1 + threadIdx.x; j < j1; j += blockDim.x) w[j] = payload_word(seed, p, j);
}

// Staging tile k of a staged request whose region starts at `reg` on every PE it touches:
// writes its share of the source part(s).  PUT/GET: bytes of one RMA tile on the source
// PE; REDUCE: the elements of one reduce tile on every member (bf16: their codes and the
// scales of their blocks); ALLTOALL: one A2A_TILE chunk of one member's source blocks.
__device__ void stage_tile(const SvArgs &a, const shmemg_req_t &r, uint64_t reg, uint32_t k) {
    uint8_t *heap = a.heap;
    const uint64_t H = a.H, seed = r.word;
    const StagedParts sp = staged_parts(r);
    switch (r.kind) {
    case SHMEMG_OP_PUT:
    case SHMEMG_OP_GET: {
        const int p = r.kind == SHMEMG_OP_PUT ? r.issuer : r.pe;
        const uint64_t b0 = (uint64_t)k * RMA_TILE, b1 = b0 + RMA_TILE < r.n ? b0 + RMA_TILE : r.n;
        stage_words(heap + (uint64_t)p * H + reg + sp.src, seed, p, b0 / 4, b1 / 4);
        break;
    }
    case SHMEMG_OP_REDUCE: {
        const uint64_t e0 = (uint64_t)k * RED_TILE, e1 = e0 + RED_TILE < r.n ? e0 + RED_TILE : r.n;
        const bool bf = r.dtype == SHMEMG_FLOAT && r.fmt == SHMEMG_FMT_BF16;
        const uint64_t es = r.dtype == SHMEMG_INT64 ? 8 : bf ? 2 : 4;
        for (int m = 0; m < r.issuer; m++) {
            const int p = r.pe + m;
            uint8_t *part = heap + (uint64_t)p * H + reg + sp.src;
            stage_words(part, seed, p, e0 * es / 4, e1 * es / 4);
            if (bf)
                stage_words(part, seed, p, (sp.scales - sp.src) / 4 + e0 / 128, (sp.scales - sp.src) / 4 + (e1 + 127) / 128);
        }
        break;
    }
    case SHMEMG_OP_ALLTOALL: {
        const uint64_t span = (uint64_t)r.issuer * r.n, per = (span + A2A_TILE - 1) / A2A_TILE;
        const int i = (int)(k / per);
        const uint64_t b0 = (k - (uint64_t)i * per) * A2A_TILE, b1 = b0 + A2A_TILE < span ? b0 + A2A_TILE : span;
        const int p = r.pe + i;
        stage_words(heap + (uint64_t)p * H + reg + sp.src, seed, p, b0 / 4, b1 / 4);
        break;
    }
    default:
        break;
    }
}

// one tile of a request (all threads of the CTA); returns this thread's checksum terms
// (AMO: thread 0 stores the fetched value through *amo_out).  Tiles below `nstage` stage
// a staged request's payload; the operation's tile k runs as tile k - nstage, its source
// in the request's region.
__device__ uint64_t run_tile(const SvArgs &a, const shmemg_req_t &r0, uint64_t dst_off, uint32_t k,
                             unsigned long long *amo_out, uint32_t nstage = 0) {
    uint8_t *heap = a.heap;
    const uint64_t H = a.H;
    shmemg_req_t r = r0;
    if (r0.flags & SHMEMG_REQ_STAGED) {
        if (k < nstage) {
            stage_tile(a, r0, dst_off, k);
            return 0;
        }
        k -= nstage;
        const StagedParts sp = staged_parts(r0);
        r.src = dst_off + sp.src;                 // fp32 / int64 reductions: in place
        r.cond = (int64_t)(dst_off + sp.scales);
    }
    switch (r.kind) {
    case SHMEMG_OP_PUT:
    case SHMEMG_OP_GET: {
        const int sp = r.kind == SHMEMG_OP_PUT ? r.issuer : r.pe, dp = r.kind == SHMEMG_OP_PUT ? r.pe : r.issuer;
        const uint64_t b0 = (uint64_t)k * RMA_TILE, b1 = b0 + RMA_TILE < r.n ? b0 + RMA_TILE : r.n;
        return copy_ck(heap + (uint64_t)dp * H + dst_off, heap + (uint64_t)sp * H + r.src, b0, b1, 0);
    }
    case SHMEMG_OP_FETCH_ADD:
    case SHMEMG_OP_COMPARE_SWAP:
    case SHMEMG_OP_FETCH_XOR: {
        if (threadIdx.x == 0) {
            const uint64_t pe = r.word / a.cfg.amo_words, idx = r.word - pe * a.cfg.amo_words;
            unsigned long long *t = (unsigned long long *)(heap + pe * H + a.cfg.amo_offset + idx * 8);
            unsigned long long old;
            if (r.kind == SHMEMG_OP_FETCH_ADD) old = atomicAdd(t, (unsigned long long)r.operand);
            else if (r.kind == SHMEMG_OP_COMPARE_SWAP) old = atomicCAS(t, (unsigned long long)r.cond, (unsigned long long)r.operand);
            else old = atomicXor(t, (unsigned long long)r.operand);
            *amo_out = old;
        }
        return 0;
    }
    case SHMEMG_OP_REDUCE: {
        const int P = r.issuer, pe0 = r.pe;
        const uint64_t e0 = (uint64_t)k * RED_TILE, e1 = e0 + RED_TILE < r.n ? e0 + RED_TILE : r.n;
        uint64_t acc = 0;
        if (r.dtype == SHMEMG_INT64) {
            for (uint64_t v = e0 / 2 + threadIdx.x; v < e1 / 2; v += blockDim.x) {
                const uint64_t off = r.src + 16 * v;
                longlong2 s = __ldcg((const longlong2 *)(heap + (uint64_t)pe0 * H + off));
                auto add = [&](const longlong2 &x) {
                    s.x = (long long)((unsigned long long)s.x + (unsigned long long)x.x);
                    s.y = (long long)((unsigned long long)s.y + (unsigned long long)x.y);
                };
                int m = 1;
                for (; m + 3 < P; m += 4) {  // four members' loads in flight
                    const longlong2 x0 = __ldcg((const longlong2 *)(heap + (uint64_t)(pe0 + m) * H + off));
                    const longlong2 x1 = __ldcg((const longlong2 *)(heap + (uint64_t)(pe0 + m + 1) * H + off));
                    const longlong2 x2 = __ldcg((const longlong2 *)(heap + (uint64_t)(pe0 + m + 2) * H + off));
                    const longlong2 x3 = __ldcg((const longlong2 *)(heap + (uint64_t)(pe0 + m + 3) * H + off));
                    add(x0);
                    add(x1);
                    add(x2);
                    add(x3);
                }
                for (; m < P; m++) add(__ldcg((const longlong2 *)(heap + (uint64_t)(pe0 + m) * H + off)));
                for (int m = 0; m < P; m++) *(longlong2 *)(heap + (uint64_t)(pe0 + m) * H + dst_off + 16 * v) = s;
                uint4 w;
                memcpy(&w, &s, 16);
                acc += ck4(w, 4 * v);
            }
        } else if (r.fmt == FMT_F32) {
            for (uint64_t v = e0 / 4 + threadIdx.x; v < e1 / 4; v += blockDim.x) {
                const float4 s = shmemg_tree_sum<float4>(heap, H, pe0, 1, P, r.src + 16 * v);
                for (int m = 0; m < P; m++) *(float4 *)(heap + (uint64_t)(pe0 + m) * H + dst_off + 16 * v) = s;
                uint4 w;
                memcpy(&w, &s, 16);
                acc += ck4(w, 4 * v);
            }
        } else {
            // bf16: eight elements per thread with 16-byte code loads, eight members'
            // codes and scales loaded ahead (sources and scales are 16-byte aligned); a
            // trailing group of four the 4-wide way
            const uint64_t v1 = e1 / 8;
            for (uint64_t v = e0 / 8 + threadIdx.x; v < v1; v += blockDim.x) {
                float4 o[2];
                qsum_wide_acc<SHMEMG_FMT_BF16>(heap, H, pe0, 1, P, r.src, (uint64_t)r.cond, 8 * v, o);
                for (int m = 0; m < P; m++) {
                    float4 *d = (float4 *)(heap + (uint64_t)(pe0 + m) * H + dst_off + 32 * v);
                    d[0] = o[0];
                    d[1] = o[1];
                }
                uint4 w0, w1;
                memcpy(&w0, &o[0], 16);
                memcpy(&w1, &o[1], 16);
                acc += ck4(w0, 8 * v) + ck4(w1, 8 * v + 4);
            }
            for (uint64_t q = 2 * v1 + threadIdx.x; q < e1 / 4; q += blockDim.x) {
                qsum4<SHMEMG_FMT_BF16>(heap, H, pe0, 1, P, dst_off, r.src, (uint64_t)r.cond, 4 * q, r.n, true);
                uint4 w = __ldcg((const uint4 *)(heap + (uint64_t)pe0 * H + dst_off + 16 * q));
                acc += ck4(w, 4 * q);
            }
        }
        return acc;
    }
    case SHMEMG_OP_ALLTOALL: {
        const int P = r.issuer, pe0 = r.pe;
        const uint64_t chunks = (r.n + A2A_TILE - 1) / A2A_TILE;
        const uint64_t pair = k / chunks, ch = k - pair * chunks;
        const int i = (int)(pair / (uint64_t)P), j = (int)(pair - (uint64_t)i * P);
        const uint64_t b0 = ch * A2A_TILE, b1 = b0 + A2A_TILE < r.n ? b0 + A2A_TILE : r.n;
        const uint64_t wbase = ((uint64_t)j * P * r.n + (uint64_t)i * r.n) / 4;
        return copy_ck(heap + (uint64_t)(pe0 + j) * H + dst_off + (uint64_t)i * r.n,
                       heap + (uint64_t)(pe0 + i) * H + r.src + (uint64_t)j * r.n, b0, b1, wbase);
    }
    default:
        return 0;
    }
}

__device__ __forceinline__ uint64_t block_sum_u64(uint64_t v) {
    __shared__ uint64_t s_part[32];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    uint64_t t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_part[w];
    __syncthreads();
    return t;  // valid in thread 0
}

// completion record to mapped host memory (thread scope); bounded wait for ring room
__device__ void write_completion(const SvArgs &a, uint64_t ticket, uint64_t t_admit, uint64_t result, int status) {
    const unsigned long long pos = atomicAdd(&a.ctl->comp_pos, 1ull);
    if (pos - *(volatile unsigned long long *)&a.ctl->consumed_cache >= a.ring_slots) {
        // ring looks full from the cached credit: ask the host how far it has read
        const uint64_t t0 = now_dev();
        for (;;) {
            const unsigned long long cons = a.host->consumed;
            if (pos - cons < a.ring_slots) {
                atomicMax(&a.ctl->consumed_cache, cons);
                break;
            }
            if (now_dev() - t0 > 2000000000ull) return;  // host stopped reading: drop the record
            __nanosleep(1000);
        }
    }
    volatile shmemg_completion_t *c = a.comp + (pos % a.ring_slots);
    c->ticket = ticket;
    c->t_admit_ns = t_admit;
    c->t_done_ns = now_dev();
    c->result = result;
    c->status = status;
    // the release orders the record's fields before its sequence number
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"((const uint32_t *)&c->seq), "r"((uint32_t)(pos + 1))
                 : "memory");
}

// ------------------------------------------------------------------ admitter
// Page bitmaps, warp-collective (all 32 lanes call with the same arguments): lane m
// handles members m, m + 32, ... of the request's PEs, so a request spread over P PEs
// costs about P/32 dependent loads or atomics per bitmap word, not P.
__device__ bool find_pages(const SvArgs &a, const Geo &g, uint32_t need, uint32_t *first, int lane) {
    if (need == 0) { *first = 0; return true; }
    if (need > a.pages_per_pe) return false;
    uint32_t run = 0;
    for (uint32_t w = 0; w < a.bm_words; w++) {
        unsigned long long mine = 0;
        for (int m = lane; m < g.count + g.count2; m += 32)
            mine |= *(volatile unsigned long long *)&a.bitmaps[(uint64_t)geo_pe(g, m) * a.bm_words + w];
        const unsigned long long occ = (unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)mine) |
                                       ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(mine >> 32)) << 32);
        for (int b = 0; b < 64; b++) {
            const uint32_t page = w * 64 + b;
            if (page >= a.pages_per_pe) return false;
            if ((occ >> b) & 1ull) {
                run = 0;
            } else if (++run == need) {
                *first = page + 1 - need;
                return true;
            }
        }
    }
    return false;
}

__device__ void mark_pages(const SvArgs &a, const Geo &g, uint32_t p0, uint32_t np, bool set, int lane) {
    for (int m = lane; m < g.count + g.count2; m += 32) {
        unsigned long long *bm = a.bitmaps + (uint64_t)geo_pe(g, m) * a.bm_words;
        for (uint32_t p = p0; p < p0 + np;) {
            const uint32_t w = p / 64, b = p % 64;
            const uint32_t nb = (64 - b) < (p0 + np - p) ? (64 - b) : (p0 + np - p);
            const unsigned long long mask = (nb == 64 ? ~0ull : ((1ull << nb) - 1)) << b;
            if (set) atomicOr(bm + w, mask);
            else atomicAnd(bm + w, ~mask);
            p += nb;
        }
    }
    __syncwarp();
}

// Admission state of the admitter (lane 0 of CTA 0's first warp).
struct AdmState {
    uint64_t fifo_tail, fifo_published;
    uint32_t rot;
};

// Publishes the slots admitted since the last flush: one GPU-scope fence orders every
// slot field and claim word before the queue tail that workers acquire.
__device__ __forceinline__ void adm_flush(const SvArgs &a, AdmState &st) {
    if (st.fifo_published == st.fifo_tail) return;
    shmemg_d_fence_gpu();
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(&a.ctl->fifo_tail), "l"((unsigned long long)st.fifo_tail)
                 : "memory");
    st.fifo_published = st.fifo_tail;
}

// Tries to admit one request: 1 = admitted (or completed with an error), 0 = no slot,
// queue room or pages yet (retry later).  Warp-collective: every lane computes the same
// verdict (lane 0's reads are broadcast); lane 0 writes the slot and the queue.
__device__ int adm_try(const SvArgs &a, AdmState &st, const shmemg_req_t &r, uint64_t now, int lane) {
    const Geo g = geometry(r, a.npes, a.H, a.cfg.amo_words);
    if (!g.valid) {
        if (lane == 0) write_completion(a, r.ticket, now, 0, SHMEMG_ERR_INVALID_ARG);
        __syncwarp();
        return 1;
    }
    const uint32_t need = (uint32_t)((g.bytes + a.cfg.page_bytes - 1) / a.cfg.page_bytes);
    if (need > a.pages_per_pe) {
        if (lane == 0) write_completion(a, r.ticket, now, 0, SHMEMG_ERR_OUT_OF_HEAP);
        __syncwarp();
        return 1;
    }
    int slot = -1;
    if (lane == 0) {
        // the queue head and the first candidate slot are read together; a slot is taken
        // only through an acquire load of its busy word (its finalizer released it)
        const uint32_t k0 = st.rot % a.nslots;
        const unsigned long long head = *(volatile unsigned long long *)&a.ctl->fifo_head;
        const uint32_t b0 = shmemg_d_ld_acquire_u32(&a.slots[k0].busy);
        if (st.fifo_tail - head < a.fifo_cap) {
            if (b0 == 0) slot = (int)k0;
            for (uint32_t i = 1; i < a.nslots && slot < 0; i++) {
                const uint32_t k = (st.rot + i) % a.nslots;
                if (shmemg_d_ld_acquire_u32(&a.slots[k].busy) == 0) slot = (int)k;
            }
        }
    }
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot < 0) return 0;
    uint32_t p0 = 0;
    if (!find_pages(a, g, need, &p0, lane)) return 0;
    if (need) shmemg_d_fence_gpu();  // page frees seen above happen before the pages' reuse
    mark_pages(a, g, p0, need, true, lane);
    SvSlot &s = a.slots[slot];
    if (lane == 0) {
        const uint32_t gen = s.gen + 1;
        s.req = r;
        s.dst_off = a.cfg.arena_offset + (uint64_t)p0 * a.cfg.page_bytes;
        s.page0 = p0;
        s.npages = need;
        s.ntiles = g.ntiles;
        s.nstage = g.nstage;
        s.staged = 0;
        s.gen = gen;
        s.done = 0;
        s.checksum = 0;
        s.t_admit = now;
        s.status = 0;
        s.busy = 1;
        // release: a worker whose fetch-and-add sees this generation also sees the fields
        // above (and the page marks, ordered before it by the warp barrier)
        asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(&s.claim), "l"((unsigned long long)gen << 32)
                     : "memory");
        atomicAdd(&a.ctl->inflight, 1ull);
        a.fifo[st.fifo_tail % a.fifo_cap] = ((unsigned long long)gen << 32) | (unsigned)slot;
        s.t_pub = now_dev();
    }
    __syncwarp();
    st.fifo_tail++;
    st.rot = (uint32_t)slot + 1;
    return 1;
}

// The admitter warp: each round it acquires the ring tail, reads up to 8 requests with
// one 16-byte system-scope load per lane (4 lanes per 64-byte request), admits them in
// order on lane 0 and publishes the batch with one fence.
// The admitter warp keeps up to PEND requests taken from the ring and admits any of
// them that fits now (oldest first), so a request waiting for pages does not hold back
// later ones; once the oldest has waited AGE_NS, only it is tried until it is admitted
// (no starvation).  Each round the warp acquires the ring tail and reads up to 8 new
// requests with one 16-byte system-scope load per lane (4 lanes per 64-byte request);
// admitted requests are published with one fence per round.
constexpr int PEND = 32;
constexpr uint64_t AGE_NS = 2000000;

__device__ void admitter_warp(const SvArgs &a) {
    __shared__ __align__(16) shmemg_req_t s_pend[PEND];  // 16-byte stores below
    __shared__ uint64_t s_since[PEND];
    __shared__ int s_ctl[2];
    __shared__ int s_npend, s_adm;
    const int lane = threadIdx.x & 31;
    uint64_t head = 0;
    AdmState st = {0, 0, 0};
    const uint64_t t_start = now_dev();
    uint64_t t_last = t_start;
    uint32_t sleep_ns = 64;
    if (lane == 0) s_npend = 0;
    __syncwarp();
    for (;;) {
        if (lane == 0) {
            const uint64_t now = now_dev();
            const uint64_t tail = shmemg_d_ld_acquire_sys_u64(&a.host->tail);
            const uint64_t room = (uint64_t)(PEND - s_npend) < 8 ? (uint64_t)(PEND - s_npend) : 8;
            int nnew = (int)(tail - head < room ? tail - head : room), stop = 0;
            if (now - t_start > a.cfg.max_ns) stop = 1;
            if (nnew == 0 && s_npend == 0 && !stop) {
                const bool idle = *(volatile unsigned long long *)&a.ctl->inflight == 0;
                if (idle && (a.host->stop || now - t_last > a.cfg.idle_ns)) stop = 1;
            }
            s_ctl[0] = nnew;
            s_ctl[1] = stop;
        }
        __syncwarp();
        const int nnew = s_ctl[0];
        if (s_ctl[1]) break;
        if (nnew > 0) {
            const int q = lane >> 2, part = lane & 3, base = s_npend;
            if (q < nnew) {
                const uint32_t *p = (const uint32_t *)(a.ring + ((head + q) % a.ring_slots)) + 4 * part;
                uint4 v;
                asm volatile("ld.relaxed.sys.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                             : "l"(p)
                             : "memory");
                reinterpret_cast<uint4 *>(&s_pend[base + q])[part] = v;
            }
            head += (uint64_t)nnew;  // every lane: the next read uses it
        }
        __syncwarp();
        int admitted = 0;
        {
            const uint64_t now = __shfl_sync(0xffffffffu, now_dev(), 0);
            if (lane == 0)
                for (int i = s_npend; i < s_npend + nnew; i++) s_since[i] = now;
            __syncwarp();
            const int n = s_npend + nnew;
            const bool aged = n > 0 && now - s_since[0] > AGE_NS;
            int k = 0;
            for (int i = 0; i < n; i++) {  // the whole warp admits, in order
                const bool try_it = !aged || i == 0;
                if (try_it && adm_try(a, st, s_pend[i], now, lane)) {
                    admitted++;
                    continue;
                }
                if (k != i && lane == 0) {
                    s_pend[k] = s_pend[i];
                    s_since[k] = s_since[i];
                }
                __syncwarp();
                k++;
            }
            if (lane == 0) s_npend = k;
            __syncwarp();
        }
        if (lane == 0) {
            const uint64_t now = now_dev();
            adm_flush(a, st);
            if (nnew > 0)
                asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"((const uint64_t *)&a.host->head), "l"(head)
                             : "memory");
            if (nnew > 0 || admitted) t_last = now;
            s_adm = admitted;
        }
        __syncwarp();
        if (nnew == 0 && s_adm == 0) {
            __nanosleep(sleep_ns);
            if (sleep_ns < 256) sleep_ns <<= 1;
        } else {
            sleep_ns = 64;
        }
    }
    if (lane == 0)
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&a.ctl->exit_flag), "r"(1u) : "memory");
}

// ------------------------------------------------------------------ workers
// Run by warp 0 of the worker whose publish completed the slot's tile count (every other
// publisher's tiles and checksum terms happen before that acq_rel add): frees the pages
// (lanes split the members), writes the completion record and releases the slot.
__device__ void finalize(const SvArgs &a, SvSlot &s, int lane) {
    const shmemg_req_t r = s.req;
    const Geo g = geometry(r, a.npes, a.H, a.cfg.amo_words);
    if (s.npages) mark_pages(a, g, s.page0, s.npages, false, lane);
    if (lane == 0) {
        write_completion(a, r.ticket, s.t_admit, s.checksum, s.status);
        atomicAdd(&a.ctl->inflight, ~0ull);  // -1
        // the release orders the page frees (warp barrier above) and the count before the
        // slot's reuse
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&s.busy), "r"(0u) : "memory");
    }
    __syncwarp();
}

// Publishes `cnt` finished tiles of slot s with their checksum terms (AMO: the fetched
// value): one acq_rel add on the tile count -- release for this CTA's tile writes
// (ordered before it by a CTA barrier) and the checksum, acquire for the other
// publishers'.  True for the publisher that completes the count (it finalizes).
__device__ __forceinline__ bool publish(const SvArgs &a, uint32_t slot, uint64_t sum, unsigned long long amo,
                                        uint32_t cnt) {
    SvSlot &s = a.slots[slot];
    const uint32_t kind = s.req.kind;
    if (kind == SHMEMG_OP_FETCH_ADD || kind == SHMEMG_OP_COMPARE_SWAP || kind == SHMEMG_OP_FETCH_XOR) s.checksum = amo;
    else atomicAdd(&s.checksum, (unsigned long long)sum);
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(&s.done), "r"(cnt) : "memory");
    return old + cnt == s.ntiles;
}

// Claims tiles [k, k + cnt) of whatever request slot s holds now: fetch-and-add of the
// chunk size on the slot's (generation, next tile) word with acquire semantics (the
// admitter published the slot with a release store of that word).  Big requests are
// claimed in chunks (about half of an even share per worker), so the claim word and
// the completion counter see few atomics; a claimed index below ntiles is always
// executed, even by a worker that came from an older queue entry of the same slot, so
// no index is lost.
__device__ __forceinline__ bool claim_tiles(const SvArgs &a, uint32_t slot, uint32_t *tile, uint32_t *cnt,
                                            shmemg_req_t *req, uint64_t *dst_off, uint32_t *nstage,
                                            uint32_t nt_seen = 0) {
    SvSlot &s = a.slots[slot];
    // a plain look first (unless the caller has just looked, and passes the tile count it
    // saw): an exhausted request costs no atomic on its busy claim line
    const uint32_t nt = nt_seen ? nt_seen : *(volatile uint32_t *)&s.ntiles;
    if (!nt_seen && (uint32_t)*(volatile unsigned long long *)&s.claim >= nt) return false;
    const uint32_t nworkers = gridDim.x - 1;
    uint32_t chunk = nt / (2 * nworkers);
    chunk = chunk < 1 ? 1 : chunk > 64 ? 64 : chunk;
    unsigned long long c;
    asm volatile("atom.acquire.gpu.global.add.u64 %0, [%1], %2;" : "=l"(c) : "l"(&s.claim), "l"((unsigned long long)chunk)
                 : "memory");
    // the request and its destination are read together with the tile count (all ordered
    // after the acquire above), so the claim costs one round trip more, not three
    const uint32_t k = (uint32_t)c, n = *(volatile uint32_t *)&s.ntiles;
    const shmemg_req_t rq = s.req;
    const uint64_t d = s.dst_off;
    const uint32_t ns = s.nstage;
    if (k < n) {
        *tile = k;
        *cnt = k + chunk <= n ? chunk : n - k;
        *req = rq;
        *dst_off = d;
        *nstage = ns;
        return true;
    }
    return false;
}

// Thread 0 of a worker about to run an operation tile of a staged request: acquire-waits
// until all `ns` staging tiles are counted (they were claimed before it, by workers that
// run them without waiting on anything); false after 10 s.
__device__ bool wait_staged(const SvArgs &a, SvSlot &s, uint32_t ns) {
    if (shmemg_d_ld_acquire_u32(&s.staged) >= ns) return true;
    const uint64_t t0 = now_dev();
    for (uint32_t sl = 32;;) {
        if (shmemg_d_ld_acquire_u32(&s.staged) >= ns) return true;
        if (now_dev() - t0 > 10000000000ull) return false;
        __nanosleep(sl);
        if (sl < 256) sl <<= 1;
    }
}

// A worker CTA.  Thread 0 claims chunks of tiles, the CTA runs them; the finished tiles
// of a slot are published together when the worker leaves the slot (its next claim there
// fails) or at once when the chunk held the slot's last tile (nobody will claim after
// it), so a worker that keeps claiming one request pays one publish for all its tiles.
// Two workers share an SM; the first on each SM (its primary) gets a head start on a newly
// queued request, so a request with fewer tiles than SMs spreads over distinct SMs
// instead of doubling up on some while others idle.  Idle workers watch only the queue
// tail (one relaxed load) until it moves.
__device__ void worker(const SvArgs &a) {
    __shared__ int s_cmd;
    __shared__ int s_fin;  // slot whose count this CTA's publish completed (warp 0 finalizes), -1 none
    __shared__ uint32_t s_slot, s_tile, s_cnt;
    __shared__ unsigned long long s_amo;
    __shared__ __align__(16) shmemg_req_t s_req;   // the claimed slot's request and destination
    __shared__ uint64_t s_dst;
    __shared__ uint32_t s_nstage;
    const uint32_t me = blockIdx.x - 1;
    bool primary = true;
    if (threadIdx.x == 0) s_fin = -1;
    if (threadIdx.x == 0) {
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        primary = atomicAdd(&a.ctl->sm_workers[smid % SV_MAX_SMID], 1u) == 0;
    }
    const uint32_t max_sleep = primary ? 256 : 1024;
    unsigned long long idle_tail = ~0ull;  // thread 0: queue tail of the last scan that found it empty
    uint32_t sleep_ns = 32;
    int sticky = -1;                    // slot of the last claim: try it again first
    uint32_t pend_cnt = 0;              // thread 0: finished, unpublished tiles of `sticky`
    uint64_t pend_sum = 0;
    unsigned long long pend_amo = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int cmd = 0;
            uint32_t tile, cnt;
            if (sticky >= 0 && claim_tiles(a, (uint32_t)sticky, &tile, &cnt, &s_req, &s_dst, &s_nstage)) {
                s_slot = (uint32_t)sticky;
                s_tile = tile;
                s_cnt = cnt;
                cmd = 1;
            } else {
                if (pend_cnt && publish(a, (uint32_t)sticky, pend_sum, pend_amo, pend_cnt))  // leaving the slot
                    s_fin = sticky;
                pend_cnt = 0;
                pend_sum = 0;
                sticky = -1;
            }
            for (int tries = 0; tries < 64 && cmd == 0; tries++) {
                if (*(volatile unsigned int *)&a.ctl->exit_flag) { cmd = -1; break; }
                if (idle_tail != ~0ull && *(volatile unsigned long long *)&a.ctl->fifo_tail == idle_tail) break;
                const unsigned long long h = shmemg_d_ld_acquire_u64((const uint64_t *)&a.ctl->fifo_head);
                const unsigned long long t = shmemg_d_ld_acquire_u64((const uint64_t *)&a.ctl->fifo_tail);
                if (h >= t) {
                    idle_tail = t;  // nothing queued: nothing new until the tail moves
                    break;
                }
                idle_tail = ~0ull;
                const uint32_t live = (uint32_t)((t - h) < WINDOW ? (t - h) : WINDOW);
                const uint32_t start = me % live;
                for (uint32_t j = 0; j < live && cmd == 0; j++) {
                    const unsigned long long pos = h + (start + j) % live;
                    const unsigned long long e = *(volatile unsigned long long *)&a.fifo[pos % a.fifo_cap];
                    const uint32_t slot = (uint32_t)e, gen = (uint32_t)(e >> 32);
                    SvSlot &s = a.slots[slot];
                    const unsigned long long c = *(volatile unsigned long long *)&s.claim;
                    const uint32_t nt = *(volatile uint32_t *)&s.ntiles;
                    if ((uint32_t)(c >> 32) != gen || (uint32_t)c >= nt) {
                        if (pos == h) atomicCAS(&a.ctl->fifo_head, h, h + 1);  // exhausted or stale head
                        continue;
                    }
                    if (!primary && now_dev() - *(volatile uint64_t *)&s.t_pub < SECONDARY_DELAY_NS) continue;
                    if (claim_tiles(a, slot, &tile, &cnt, &s_req, &s_dst, &s_nstage, nt)) {   // claim word and tile count read just above
                        s_slot = slot;
                        s_tile = tile;
                        s_cnt = cnt;
                        sticky = (int)slot;
                        cmd = 1;
                    }
                }
            }
            s_cmd = cmd;
        }
        __syncthreads();
        if (s_fin >= 0) {  // warp 0 finalizes the request this CTA completed
            if (threadIdx.x < 32) finalize(a, a.slots[s_fin], threadIdx.x);
            __syncthreads();
            if (threadIdx.x == 0) s_fin = -1;
        }
        const int cmd = s_cmd;
        if (cmd < 0) break;
        if (cmd == 0) {
            __syncthreads();
            __nanosleep(sleep_ns);
            if (sleep_ns < max_sleep) sleep_ns <<= 1;
            continue;
        }
        sleep_ns = 32;
        SvSlot &s = a.slots[s_slot];
        const shmemg_req_t r = s_req;
        const uint64_t dst_off = s_dst;
        const uint32_t t0 = s_tile, cnt = s_cnt, ns = s_nstage;
        uint64_t part = 0;
        uint32_t staged_here = 0;  // staging tiles of this chunk not yet counted in s.staged
        for (uint32_t k = 0; k < cnt; k++) {
            const uint32_t tk = t0 + k;
            if (ns && tk >= ns && (k == 0 || tk == ns)) {
                // the operation's first tile in this chunk: count this chunk's staging
                // tiles (written before the barrier that ended each), then wait until
                // every staging tile of the request is written
                if (threadIdx.x == 0) {
                    if (staged_here)
                        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&s.staged), "r"(staged_here) : "memory");
                    if (!wait_staged(a, s, ns)) s.status = SHMEMG_ERR_TIMEOUT;
                }
                staged_here = 0;
                __syncthreads();
            }
            part += run_tile(a, r, dst_off, tk, &s_amo, ns);
            __syncthreads();  // (an AMO's fetched value is in s_amo)
            if (tk < ns) staged_here++;
        }
        if (staged_here && threadIdx.x == 0)
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&s.staged), "r"(staged_here) : "memory");
        const uint64_t sum = block_sum_u64(part);  // ends with a CTA barrier: the tiles are written
        if (threadIdx.x == 0) {
            pend_sum += sum;
            pend_amo = s_amo;
            pend_cnt += cnt;
            if (t0 + cnt >= s.ntiles) {  // the slot's last tile: nobody claims after this chunk
                if (pend_cnt == s.ntiles) {
                    // this worker ran every tile of the request: nobody else publishes,
                    // so its result goes straight to the slot (read by warp 0 of this CTA
                    // after the barrier below) without the completion counter's atomic
                    const uint32_t kind = s_req.kind;
                    s.checksum = kind == SHMEMG_OP_FETCH_ADD || kind == SHMEMG_OP_COMPARE_SWAP ||
                                         kind == SHMEMG_OP_FETCH_XOR
                                     ? pend_amo
                                     : pend_sum;
                    s_fin = (int)s_slot;
                } else if (publish(a, s_slot, pend_sum, pend_amo, pend_cnt)) {
                    s_fin = (int)s_slot;
                }
                pend_cnt = 0;
                pend_sum = 0;
                sticky = -1;
            }
        }
        __syncthreads();
        if (s_fin >= 0) {
            if (threadIdx.x < 32) finalize(a, a.slots[s_fin], threadIdx.x);
            __syncthreads();
            if (threadIdx.x == 0) s_fin = -1;
            __syncthreads();
        }
    }
    // (no unpublished tiles can remain here: the kernel exits only once nothing is in flight)
}

__global__ void __launch_bounds__(SRV_THREADS, 2) k_server(SvArgs a) {
    if (blockIdx.x == 0) {
        if (threadIdx.x < 32) admitter_warp(a);
        return;
    }
    worker(a);
}

// ------------------------------------------------------------------ plain path
struct PlainScratch {
    unsigned long long checksum, amo;
    unsigned int done, pad;
    uint64_t t_start;
};

// Tiles [lo, hi) of request r, grid-stride.  A staged request runs as two launches on one
// stream: its staging tiles, then its operation tiles (final = 1: that launch's last CTA
// writes the completion record).
__global__ void __launch_bounds__(SV_THREADS, 2) k_plain(SvArgs a, shmemg_req_t r, uint32_t lo, uint32_t hi,
                                                      uint32_t nstage, int final, int status, PlainScratch *sc,
                                                      shmemg_completion_t *rec) {
    __shared__ unsigned long long s_amo;
    if (lo == 0 && blockIdx.x == 0 && threadIdx.x == 0) sc->t_start = now_dev();
    uint64_t part = 0;
    if (status == SHMEMG_SUCCESS)
        for (uint32_t k = lo + blockIdx.x; k < hi; k += gridDim.x) {
            part += run_tile(a, r, a.cfg.arena_offset, k, &s_amo, nstage);
            __syncthreads();
            if (threadIdx.x == 0 && (r.kind == SHMEMG_OP_FETCH_ADD || r.kind == SHMEMG_OP_COMPARE_SWAP ||
                                     r.kind == SHMEMG_OP_FETCH_XOR))
                sc->amo = s_amo;
        }
    const uint64_t sum = block_sum_u64(part);
    if (threadIdx.x == 0) {
        atomicAdd(&sc->checksum, (unsigned long long)sum);
        shmemg_d_fence_gpu();
        const bool last = atomicAdd(&sc->done, 1u) == gridDim.x - 1;
        if (last && !final) {
            sc->done = 0;  // the staging launch: the next launch on the stream counts anew
            shmemg_d_fence_gpu();
        } else if (last) {
            shmemg_d_fence_gpu();
            const bool amo = r.kind == SHMEMG_OP_FETCH_ADD || r.kind == SHMEMG_OP_COMPARE_SWAP ||
                             r.kind == SHMEMG_OP_FETCH_XOR;
            volatile shmemg_completion_t *c = rec;
            c->ticket = r.ticket;
            c->t_admit_ns = sc->t_start;
            c->result = amo ? sc->amo : sc->checksum;
            c->status = status;
            c->t_done_ns = now_dev();
            c->seq = 1;
            sc->checksum = 0;
            sc->amo = 0;
            sc->done = 0;
            shmemg_d_fence_sys();
        }
    }
}

__global__ void k_stamp(uint64_t *out) { *out = shmemg_d_globaltimer(); }

static uint64_t host_ns() {
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (uint64_t)t.tv_sec * 1000000000ull + (uint64_t)t.tv_nsec;
}

static int cfg_check(const shmemg_server_cfg_t &c0, shmemg_server_cfg_t *out) {
    State &S = st();
    shmemg_server_cfg_t c = c0;
    if (c.page_bytes == 0) c.page_bytes = 65536;
    if (c.ring_slots == 0) c.ring_slots = 65536;
    if (c.max_inflight == 0) c.max_inflight = 1024;
    if (c.idle_ns == 0) c.idle_ns = 60ull * 1000000000ull;
    if (c.max_ns == 0) c.max_ns = 600ull * 1000000000ull;
    if (c.page_bytes % 256 || c.ring_slots < 2 || (c.ring_slots & (c.ring_slots - 1)) || c.max_inflight < 1)
        return SHMEMG_ERR_INVALID_ARG;
    if (c.arena_offset % 256 || c.arena_offset > S.H || c.arena_bytes > S.H - c.arena_offset) return SHMEMG_ERR_INVALID_ARG;
    if (c.arena_bytes / c.page_bytes > 4096) return SHMEMG_ERR_INVALID_ARG;
    if (c.amo_words && (c.amo_offset % 8 || c.amo_offset > S.H || c.amo_words * 8 > S.H - c.amo_offset))
        return SHMEMG_ERR_INVALID_ARG;
    *out = c;
    return SHMEMG_SUCCESS;
}

}  // namespace shmemg

using namespace shmemg;

struct shmemg_server_s {
    SvArgs args;
    SvHost *host = nullptr;            // mapped host control
    shmemg_req_t *ring = nullptr;      // mapped host ring
    shmemg_completion_t *comp = nullptr;
    void *dev_mem = nullptr;           // bitmaps, slots, fifo, ctl
    uint64_t tail = 0, comp_next = 0, ticket = 0;
    cudaStream_t stream = nullptr;
};

static void server_free(shmemg_server_s *s) {
    if (s->dev_mem) cudaFree(s->dev_mem);
    if (s->host) cudaFreeHost(s->host);
    if (s->ring) cudaFreeHost(s->ring);
    if (s->comp) cudaFreeHost(s->comp);
    delete s;
}

extern "C" {

int shmemg_server_start(const shmemg_server_cfg_t *cfg_in, void *stream, shmemg_server_t *out) {
    if (int rc = check_init()) return rc;
    if (!cfg_in || !out) return SHMEMG_ERR_INVALID_ARG;
    State &S = st();
    shmemg_server_cfg_t cfg;
    if (int rc = cfg_check(*cfg_in, &cfg)) return rc;
    auto *s = new shmemg_server_s();
    SvArgs &a = s->args;
    memset(&a, 0, sizeof(a));
    a.heap = S.heap;
    a.H = S.H;
    a.npes = S.npes;
    a.cfg = cfg;
    a.pages_per_pe = (uint32_t)(cfg.arena_bytes / cfg.page_bytes);
    a.bm_words = (a.pages_per_pe + 63) / 64;
    a.nslots = (uint32_t)cfg.max_inflight;
    a.fifo_cap = 1;
    while (a.fifo_cap < 2 * a.nslots) a.fifo_cap <<= 1;
    a.ring_slots = (uint32_t)cfg.ring_slots;
    size_t bm_bytes = (size_t)S.npes * (a.bm_words ? a.bm_words : 1) * 8;
    size_t off_slots = (bm_bytes + 255) & ~(size_t)255;
    size_t off_fifo = off_slots + (((size_t)a.nslots * sizeof(SvSlot) + 255) & ~(size_t)255);
    size_t off_ctl = off_fifo + (((size_t)a.fifo_cap * 8 + 255) & ~(size_t)255);
    size_t total = off_ctl + sizeof(SvCtl);
    int rc = cuda_rc(cudaMalloc(&s->dev_mem, total));
    if (!rc) rc = cuda_rc(cudaMemset(s->dev_mem, 0, total));
    if (!rc) rc = cuda_rc(cudaHostAlloc((void **)&s->host, sizeof(SvHost), cudaHostAllocMapped));
    if (!rc) rc = cuda_rc(cudaHostAlloc((void **)&s->ring, sizeof(shmemg_req_t) * a.ring_slots, cudaHostAllocMapped));
    if (!rc) rc = cuda_rc(cudaHostAlloc((void **)&s->comp, sizeof(shmemg_completion_t) * a.ring_slots, cudaHostAllocMapped));
    if (rc) { server_free(s); return rc; }
    memset((void *)s->host, 0, sizeof(SvHost));
    memset(s->ring, 0, sizeof(shmemg_req_t) * a.ring_slots);
    memset(s->comp, 0, sizeof(shmemg_completion_t) * a.ring_slots);
    uint8_t *d = (uint8_t *)s->dev_mem;
    a.bitmaps = (unsigned long long *)d;
    a.slots = (SvSlot *)(d + off_slots);
    a.fifo = (unsigned long long *)(d + off_fifo);
    a.ctl = (SvCtl *)(d + off_ctl);
    void *p;
    if ((rc = cuda_rc(cudaHostGetDevicePointer(&p, (void *)s->host, 0)))) { server_free(s); return rc; }
    a.host = (SvHost *)p;
    if ((rc = cuda_rc(cudaHostGetDevicePointer(&p, s->ring, 0)))) { server_free(s); return rc; }
    a.ring = (shmemg_req_t *)p;
    if ((rc = cuda_rc(cudaHostGetDevicePointer(&p, s->comp, 0)))) { server_free(s); return rc; }
    a.comp = (shmemg_completion_t *)p;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_server, SRV_THREADS, 0);
    int cap = per_sm * S.sm_count;
    int workers = cfg.workers > 0 ? cfg.workers : cap - 1;
    if (workers < 1 || workers + 1 > cap) { server_free(s); return SHMEMG_ERR_UNSUPPORTED; }
    s->stream = to_stream(stream);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(workers + 1);
    lc.blockDim = dim3(SRV_THREADS);
    lc.stream = s->stream;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeCooperative;
    at.val.cooperative = 1;
    lc.attrs = &at;
    lc.numAttrs = 1;
    void *kargs[] = {(void *)&a};
    if ((rc = cuda_rc(cudaLaunchKernelExC(&lc, (const void *)k_server, kargs)))) { server_free(s); return rc; }
    *out = s;
    return SHMEMG_SUCCESS;
}

int shmemg_server_submit(shmemg_server_t s, const shmemg_req_t *req, uint64_t *ticket) {
    if (!s || !req) return SHMEMG_ERR_INVALID_ARG;
    const uint64_t head = __atomic_load_n(&s->host->head, __ATOMIC_ACQUIRE);
    if (s->tail - head >= s->args.ring_slots) return SHMEMG_ERR_BUSY;
    shmemg_req_t r = *req;
    r.ticket = s->ticket++;
    s->ring[s->tail % s->args.ring_slots] = r;
    s->tail++;
    __atomic_store_n(&s->host->tail, s->tail, __ATOMIC_RELEASE);
    if (ticket) *ticket = r.ticket;
    return SHMEMG_SUCCESS;
}

int shmemg_server_feed(shmemg_server_t s, const shmemg_req_t *reqs, int count, const uint64_t *arrival_ns,
                       uint64_t *t0_ns) {
    if (!s || count < 0 || (count && (!reqs || !arrival_ns))) return SHMEMG_ERR_INVALID_ARG;
    const uint64_t t0 = host_ns();
    if (t0_ns) *t0_ns = t0;
    for (int i = 0; i < count; i++) {
        const uint64_t target = t0 + arrival_ns[i];
        while (host_ns() < target) {
        }
        const uint64_t give_up = host_ns() + 60ull * 1000000000ull;
        while (shmemg_server_submit(s, &reqs[i], nullptr) == SHMEMG_ERR_BUSY) {
            if (host_ns() > give_up) return SHMEMG_ERR_TIMEOUT;
        }
    }
    return SHMEMG_SUCCESS;
}

int shmemg_server_poll(shmemg_server_t s, shmemg_completion_t *out, int max, int *got) {
    if (!s || !got || max < 0 || (max && !out)) return SHMEMG_ERR_INVALID_ARG;
    int n = 0;
    while (n < max) {
        shmemg_completion_t *c = s->comp + (s->comp_next % s->args.ring_slots);
        const uint32_t seq = __atomic_load_n(&c->seq, __ATOMIC_ACQUIRE);
        if (seq != (uint32_t)(s->comp_next + 1)) break;
        out[n++] = *c;
        s->comp_next++;
    }
    __atomic_store_n(&s->host->consumed, s->comp_next, __ATOMIC_RELEASE);
    *got = n;
    return SHMEMG_SUCCESS;
}

int shmemg_server_stop(shmemg_server_t s) {
    if (!s) return SHMEMG_ERR_INVALID_ARG;
    __atomic_store_n(&s->host->stop, 1u, __ATOMIC_RELEASE);
    const uint64_t give_up = host_ns() + 60ull * 1000000000ull;
    int rc = SHMEMG_SUCCESS;
    for (;;) {
        // keep reading completions so a kernel waiting for ring room can finish
        shmemg_completion_t tmp[256];
        int got = 0;
        shmemg_server_poll(s, tmp, 256, &got);
        cudaError_t e = cudaStreamQuery(s->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) { rc = cuda_rc(e); break; }
        if (host_ns() > give_up) return SHMEMG_ERR_TIMEOUT;  // kernel still running: keep its memory
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    server_free(s);
    return rc;
}

int shmemg_request_run(const shmemg_req_t *req, const shmemg_server_cfg_t *cfg_in, shmemg_completion_t *rec,
                       void *stream) {
    if (int rc = check_init()) return rc;
    if (!req || !cfg_in || !rec) return SHMEMG_ERR_INVALID_ARG;
    State &S = st();
    shmemg_server_cfg_t cfg;
    if (int rc = cfg_check(*cfg_in, &cfg)) return rc;
    SvArgs a;
    memset(&a, 0, sizeof(a));
    a.heap = S.heap;
    a.H = S.H;
    a.npes = S.npes;
    a.cfg = cfg;
    const Geo g = geometry(*req, S.npes, S.H, cfg.amo_words);
    int status = g.valid ? SHMEMG_SUCCESS : SHMEMG_ERR_INVALID_ARG;
    if (g.valid && g.bytes > cfg.arena_bytes) status = SHMEMG_ERR_OUT_OF_HEAP;
    PlainScratch *sc = (PlainScratch *)(S.base + SHMEMG_SCRATCH_OFF + SCR_WORK) + (S.call_seq++ % 1024);
    const uint32_t cap = (uint32_t)ctas_for((const void *)k_plain, SV_THREADS, 0);
    auto grid_for = [&](uint32_t tiles) { return (int)(tiles < cap ? (tiles ? tiles : 1) : cap); };
    SvArgs ka = a;
    const uint32_t ns = status == SHMEMG_SUCCESS ? g.nstage : 0;
    if (ns) {  // the staged payload first, then the operation
        k_plain<<<grid_for(ns), SV_THREADS, 0, to_stream(stream)>>>(ka, *req, 0, ns, ns, 0, status, sc, rec);
        if (int rc = cuda_rc(cudaGetLastError())) return rc;
    }
    k_plain<<<grid_for(g.ntiles - ns), SV_THREADS, 0, to_stream(stream)>>>(ka, *req, ns, g.ntiles, ns, 1, status, sc,
                                                                           rec);
    return cuda_rc(cudaGetLastError());
}

int shmemg_plain_feed(const shmemg_req_t *reqs, int count, const uint64_t *arrival_ns, const shmemg_server_cfg_t *cfg,
                      shmemg_completion_t *recs, void *stream, uint64_t *t0_ns) {
    if (int rc = check_init()) return rc;
    if (count < 0 || (count && (!reqs || !arrival_ns || !recs)) || !cfg) return SHMEMG_ERR_INVALID_ARG;
    const uint64_t t0 = host_ns();
    if (t0_ns) *t0_ns = t0;
    for (int i = 0; i < count; i++) {
        const uint64_t target = t0 + arrival_ns[i];
        while (host_ns() < target) {
        }
        shmemg_req_t r = reqs[i];
        r.ticket = (uint64_t)i;
        if (int rc = shmemg_request_run(&r, cfg, recs + i, stream)) return rc;
    }
    return SHMEMG_SUCCESS;
}

int shmemg_clock_offset(int rounds, int64_t *offset_ns, uint64_t *err_ns) {
    if (rounds < 1 || !offset_ns || !err_ns) return SHMEMG_ERR_INVALID_ARG;
    uint64_t *d = nullptr;
    int rc = cuda_rc(cudaHostAlloc((void **)&d, 8, cudaHostAllocMapped));
    if (rc) return rc;
    uint64_t *dd = nullptr;
    cudaHostGetDevicePointer((void **)&dd, d, 0);
    uint64_t best = ~0ull;
    for (int i = 0; i < rounds; i++) {
        const uint64_t h0 = host_ns();
        k_stamp<<<1, 1>>>(dd);
        if ((rc = cuda_rc(cudaDeviceSynchronize()))) break;
        const uint64_t h1 = host_ns();
        if (h1 - h0 < best) {
            best = h1 - h0;
            *offset_ns = (int64_t)(*(volatile uint64_t *)d - (h0 + (h1 - h0) / 2));
        }
    }
    cudaFreeHost(d);
    *err_ns = best / 2;
    return rc;
}

}  // extern "C"
