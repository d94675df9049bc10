// Host-issued, stream-triggered operations (paper Sec. 6.3: "an implementation may
// use internal GPU kernels to accelerate a host-issued or stream-triggered
// operation"): RMA, AMOs, put-with-signal, wait, and the team collectives, each one
// full-grid kernel on the caller's stream.
//
// Data movement is split into work items of one chunk (blockDim x 4 vectors); a CTA
// takes items round-robin, each thread keeps its 4 vector loads in flight before it
// stores them (to one destination, or to every team member for broadcast/fcollect).
// Reductions use a slice-owner schedule: a thread owns a vector of elements, reads it
// from every member, combines, and writes the result to every member.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "internal.h"

namespace shmemg {

enum XKind { X_COPY = 0, X_A2A = 1, X_BCAST = 2, X_FCOLLECT = 3 };
constexpr int XFER_THREADS = 512;
constexpr int XFER_U = 4;
constexpr int RED_THREADS = 256;
constexpr int RED_U = 2;

struct Xfer {
    uint8_t *heap;
    uint64_t H;
    int kind;
    int start, stride, size, gstride;  // team; blockIdx.y = group
    int root;
    int dst_pe, src_pe;                // X_COPY
    uint64_t dst_off, src_off;
    uint64_t seg_vec;                  // vectors per segment
    uint64_t chunk_vec;                // vectors per item
    uint64_t chunks_per_seg;
    uint64_t nitems;                   // items per group
    int mgroups;                       // broadcast / fcollect: destination members split over this many items
};

// Item -> (segment, chunk, member group); a replicating item stores to members
// [mg*size/mgroups, (mg+1)*size/mgroups) of the team.
struct XItem {
    uint64_t seg, ch;
    int r0, r1;
};
__device__ __forceinline__ XItem xitem(const Xfer &x, uint64_t item) {
    XItem t;
    const uint64_t mg = item % (uint64_t)x.mgroups, rest = item / (uint64_t)x.mgroups;
    t.seg = rest / x.chunks_per_seg;
    t.ch = rest - t.seg * x.chunks_per_seg;
    t.r0 = (int)(mg * (uint64_t)x.size / (uint64_t)x.mgroups);
    t.r1 = (int)((mg + 1) * (uint64_t)x.size / (uint64_t)x.mgroups);
    return t;
}

template <typename V>
__device__ __forceinline__ void xfer_items(const Xfer &x, uint64_t first, uint64_t step) {
    const int grp = blockIdx.y;
    const int base_pe = x.start + grp * x.gstride;
    for (uint64_t item = first; item < x.nitems; item += step) {
        const XItem it = xitem(x, item);
        const uint64_t seg = it.seg, ch = it.ch;
        uint64_t v0 = ch * x.chunk_vec;
        uint64_t nv = x.seg_vec - v0 < x.chunk_vec ? x.seg_vec - v0 : x.chunk_vec;
        const uint64_t segb = x.seg_vec * sizeof(V);
        const V *src;
        V *dst = nullptr;
        uint64_t dst_off = x.dst_off;
        bool replicate = false;
        if (x.kind == X_COPY) {
            src = (const V *)(x.heap + (uint64_t)x.src_pe * x.H + x.src_off);
            dst = (V *)(x.heap + (uint64_t)x.dst_pe * x.H + x.dst_off);
        } else if (x.kind == X_A2A) {
            int i = (int)(seg / (uint64_t)x.size), j = (int)(seg - (uint64_t)i * x.size);
            src = (const V *)(x.heap + (uint64_t)(base_pe + i * x.stride) * x.H + x.src_off + (uint64_t)j * segb);
            dst = (V *)(x.heap + (uint64_t)(base_pe + j * x.stride) * x.H + x.dst_off + (uint64_t)i * segb);
        } else if (x.kind == X_BCAST) {
            src = (const V *)(x.heap + (uint64_t)(base_pe + x.root * x.stride) * x.H + x.src_off);
            replicate = true;
        } else {  // X_FCOLLECT: source = member seg, placed at block seg of every dst
            src = (const V *)(x.heap + (uint64_t)(base_pe + (int)seg * x.stride) * x.H + x.src_off);
            dst_off = x.dst_off + seg * segb;
            replicate = true;
        }
        V buf[XFER_U];
#pragma unroll
        for (int u = 0; u < XFER_U; u++) {
            uint64_t idx = threadIdx.x + (uint64_t)u * blockDim.x;
            if (idx < nv) buf[u] = shmemg_ld_cg(src + v0 + idx);
        }
        if (!replicate) {
#pragma unroll
            for (int u = 0; u < XFER_U; u++) {
                uint64_t idx = threadIdx.x + (uint64_t)u * blockDim.x;
                if (idx < nv) dst[v0 + idx] = buf[u];
            }
        } else {
            for (int r = it.r0; r < it.r1; r++) {
                V *d = (V *)(x.heap + (uint64_t)(base_pe + r * x.stride) * x.H + dst_off);
#pragma unroll
                for (int u = 0; u < XFER_U; u++) {
                    uint64_t idx = threadIdx.x + (uint64_t)u * blockDim.x;
                    if (idx < nv) d[v0 + idx] = buf[u];
                }
            }
        }
    }
}

template <typename V>
__global__ void __launch_bounds__(XFER_THREADS) k_xfer(Xfer x) { xfer_items<V>(x, blockIdx.x, gridDim.x); }

// ------------------------------------------------------------------ bulk (TMA) variant
// One thread per CTA streams the CTA's items (chunks of XB_CHUNK bytes) through an
// XB_STAGES-deep shared-memory ring: a bulk load per chunk, then one bulk store (copy,
// alltoall) or one per team member (broadcast, fcollect) from the same stage.
constexpr int XB_STAGES = 6;
constexpr uint32_t XB_CHUNK = 32u << 10;
constexpr uint32_t XB_SMEM = XB_STAGES * XB_CHUNK;

struct XChunk {
    const uint8_t *src;
    uint8_t *dst;        // single destination (copy, alltoall)
    uint64_t dst_off;    // replicate: byte offset inside the partitions of members [r0, r1)
    uint32_t bytes;
    bool replicate;
    int r0, r1;
};

__device__ __forceinline__ XChunk xchunk(const Xfer &x, uint64_t item, int base_pe) {
    XChunk c;
    const XItem it = xitem(x, item);
    const uint64_t seg = it.seg, ch = it.ch;
    c.r0 = it.r0;
    c.r1 = it.r1;
    const uint64_t segb = x.seg_vec, off = ch * XB_CHUNK;
    c.bytes = (uint32_t)(segb - off < XB_CHUNK ? segb - off : XB_CHUNK);
    c.replicate = false;
    c.dst = nullptr;
    c.dst_off = 0;
    if (x.kind == X_COPY) {
        c.src = x.heap + (uint64_t)x.src_pe * x.H + x.src_off + off;
        c.dst = x.heap + (uint64_t)x.dst_pe * x.H + x.dst_off + off;
    } else if (x.kind == X_A2A) {
        const int i = (int)(seg / (uint64_t)x.size), j = (int)(seg - (uint64_t)i * x.size);
        c.src = x.heap + (uint64_t)(base_pe + i * x.stride) * x.H + x.src_off + (uint64_t)j * segb + off;
        c.dst = x.heap + (uint64_t)(base_pe + j * x.stride) * x.H + x.dst_off + (uint64_t)i * segb + off;
    } else if (x.kind == X_BCAST) {
        c.src = x.heap + (uint64_t)(base_pe + x.root * x.stride) * x.H + x.src_off + off;
        c.dst_off = x.dst_off + off;
        c.replicate = true;
    } else {
        c.src = x.heap + (uint64_t)(base_pe + (int)seg * x.stride) * x.H + x.src_off + off;
        c.dst_off = x.dst_off + seg * segb + off;
        c.replicate = true;
    }
    return c;
}

__global__ void __launch_bounds__(32) k_xfer_bulk(Xfer x, uint8_t *state, uint64_t timeout_ns) {
    extern __shared__ __align__(128) uint8_t ring[];
    __shared__ __align__(8) uint64_t bars[XB_STAGES];
    if (threadIdx.x != 0) return;
    const int base_pe = x.start + blockIdx.y * x.gstride;
    if (x.nitems <= blockIdx.x) return;
    const uint64_t count = (x.nitems - blockIdx.x + gridDim.x - 1) / gridDim.x;
    for (int s = 0; s < XB_STAGES; s++)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shmemg_smem_u32(&bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    for (uint64_t j = 0; j < count && j < XB_STAGES; j++) {
        const XChunk c = xchunk(x, blockIdx.x + j * gridDim.x, base_pe);
        shmemg_bulk_load(ring + j * XB_CHUNK, c.src, c.bytes, &bars[j]);
    }
    for (uint64_t j = 0; j < count; j++) {
        const uint32_t s = (uint32_t)(j % XB_STAGES);
        if (!shmemg_mbar_wait(&bars[s], (uint32_t)((j / XB_STAGES) & 1), timeout_ns)) {
            // no load of the ring may still be writing shared memory when the CTA exits
            const bool drained = shmemg_bulk_drain_loads(bars, XB_STAGES, j, count, timeout_ns);
            int *st = (int *)(state + SHMEMG_STATUS_OFF);
            if (atomicCAS(st, 0, SHMEMG_ERR_TIMEOUT) == 0)
                *(volatile int64_t *)(state + SHMEMG_STATUS_OFF + 8) = drained ? -3 : -4;
            break;
        }
        const XChunk c = xchunk(x, blockIdx.x + j * gridDim.x, base_pe);
        uint8_t *stage = ring + (uint64_t)s * XB_CHUNK;
        if (!c.replicate) {
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(c.dst),
                         "r"(shmemg_smem_u32(stage)), "r"(c.bytes)
                         : "memory");
        } else {
            for (int r = c.r0; r < c.r1; r++) {
                uint8_t *d = x.heap + (uint64_t)(base_pe + r * x.stride) * x.H + c.dst_off;
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(d),
                             "r"(shmemg_smem_u32(stage)), "r"(c.bytes)
                             : "memory");
            }
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        if (j + XB_STAGES < count) {
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            const XChunk n2 = xchunk(x, blockIdx.x + (j + XB_STAGES) * gridDim.x, base_pe);
            shmemg_bulk_load(stage, n2.src, n2.bytes, &bars[s]);
        }
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// put-with-signal: the copy, then the last CTA to finish releases the signal
template <typename V>
__global__ void __launch_bounds__(XFER_THREADS) k_put_signal(Xfer x, uint64_t *sig, uint64_t val, int op,
                                                             uint32_t *done) {
    xfer_items<V>(x, blockIdx.x, gridDim.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        shmemg_d_fence_gpu();
        uint32_t d = atomicAdd(done, 1u);
        if (d == gridDim.x - 1) {
            *done = 0;
            shmemg_d_fence_gpu();
            shmemg_d_signal_op(sig, val, op);
        }
    }
}

// ------------------------------------------------------------------ reductions
struct Red {
    uint8_t *heap;
    uint64_t H;
    int start, stride, size, gstride;
    uint64_t dst_off, src_off;
    uint64_t nvec;        // vectors (V) per member
    uint64_t chunk_vec;
    uint64_t nitems;
    uint32_t rb_chunk, rb_stages;  // k_reduce_bulk: bytes per member per chunk, ring stages
};

template <typename T, typename V, int OP>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(Red x) {
    const int pe0 = x.start + blockIdx.y * x.gstride;
    const shmemg_group g = {threadIdx.x, blockDim.x};
    for (uint64_t item = blockIdx.x; item < x.nitems; item += gridDim.x) {
        const uint64_t v0 = item * x.chunk_vec;
        const uint64_t v1 = v0 + x.chunk_vec < x.nvec ? v0 + x.chunk_vec : x.nvec;
        shmemg_d_reduce_vecs<T, V, OP>(g, x.heap, x.H, pe0, x.stride, x.size, x.dst_off, x.src_off, v0, v1);
    }
}

// Integer sum / max / min of few vectors per member: G threads share a 16-byte vector,
// each combining the members sub, sub + G, ... (integer combining is exact in any order),
// the G partial results meet by warp shuffles, and the G threads store the result to every
// G-th member.  A launch of few vectors keeps G times as many loads in flight and needs
// P / (8G) dependent rounds instead of P / 8.  Requires P >= G.
template <typename T, typename V, int OP, int G>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_split(Red x) {
    constexpr int NL = sizeof(V) / sizeof(T);
    const int pe0 = x.start + blockIdx.y * x.gstride;
    const int sub = (int)(threadIdx.x % G);
    const uint64_t per_cta = blockDim.x / G;
    auto member = [&](int r, uint64_t off) {
        return shmemg_ld_cg((const V *)(x.heap + (uint64_t)(pe0 + r * x.stride) * x.H + off));
    };
    auto comb = [&](V &a, const V &b) {
#pragma unroll
        for (int l = 0; l < NL; l++)
            reinterpret_cast<T *>(&a)[l] = shmemg_comb<T>(reinterpret_cast<T *>(&a)[l], reinterpret_cast<const T *>(&b)[l], OP);
    };
    // warp-uniform loop: every lane runs every round (lanes past the end load vector 0 and
    // store nothing), so the shuffles always see full warps
    for (uint64_t vb = blockIdx.x * per_cta; vb < x.nvec; vb += gridDim.x * per_cta) {
        const uint64_t vi = vb + threadIdx.x / G;
        const bool act = vi < x.nvec;
        const uint64_t off = x.src_off + (act ? vi : 0) * sizeof(V);
        V acc = member(sub, off);
        int r = sub + G;
        for (; r + 7 * G < x.size; r += 8 * G) {  // eight members' loads in flight
            V v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) v[u] = member(r + u * G, off);
#pragma unroll
            for (int u = 0; u < 8; u++) comb(acc, v[u]);
        }
        for (; r < x.size; r += G) comb(acc, member(r, off));
#pragma unroll
        for (int m = G / 2; m > 0; m >>= 1) {
            V o;
            if constexpr (sizeof(T) == 8) {
#pragma unroll
                for (int l = 0; l < NL; l++)
                    reinterpret_cast<long long *>(&o)[l] = __shfl_xor_sync(0xffffffffu, reinterpret_cast<long long *>(&acc)[l], m);
            } else {
#pragma unroll
                for (int l = 0; l < NL; l++)
                    reinterpret_cast<int *>(&o)[l] = __shfl_xor_sync(0xffffffffu, reinterpret_cast<int *>(&acc)[l], m);
            }
            comb(acc, o);
        }
        if (act)
            for (int q = sub; q < x.size; q += G)
                *(V *)(x.heap + (uint64_t)(pe0 + q * x.stride) * x.H + x.dst_off + vi * sizeof(V)) = acc;
    }
}

// Integer sum / max / min over many vectors per member, one CTA per SM: the CTA streams
// its chunks of the members' slices (x.rb_chunk bytes of each member per chunk) through an
// x.rb_stages-deep shared-memory ring.  The lanes of warp 0 issue the chunk's P bulk loads
// (one per member, all completing on the stage's mbarrier); the threads combine a stage
// column by column (a column is one 16-byte vector; the members are split over `nparts`
// thread groups whose partial results meet in shared memory), and each group stores the
// result to its share of the members.  The loads of later chunks are in flight while
// earlier chunks are combined and stored, so reads and writes overlap from the first chunk
// on, which the one-vector-per-thread form does not do at a few chunks per CTA.
//
// Measured on GB300 (see rb_shape): a bulk copy costs the SM's copy engine about 65-70
// cycles whatever its size below a few KiB, so the per-member pieces must be >= 1 KiB to
// keep the engine under its limit at the HBM rate; three stages of P x 1 KiB fill the
// 192 KiB ring at P = 64.  Teams of 48..64 members with 128 KiB .. 16 MiB per member take
// the ring: at 64 members it measured 1.03-1.4x the register form from 128 KiB to 8 MiB per
// member, equal at 16 MiB, and from 1% faster to 3% slower above (int64 max the slowest).  Smaller teams with wider pieces measured slower than the register form above
// 512 KiB per member; larger teams (512 B pieces) are bound by the copy engine.
constexpr int RB_THREADS = 256;
constexpr int RB_MAX_STAGES = 4;
constexpr uint32_t RB_RING = 192u << 10;
constexpr uint32_t RB_SMEM = RB_RING + 2 * RB_THREADS * 16;
constexpr uint64_t RB_MAX_BYTES = 16ull << 20;  // per member

// bulk load of `bytes` into shared memory, completing on `bar` (whose expected byte count
// the caller has already raised)
__device__ __forceinline__ void rb_load(void *smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     shmemg_smem_u32(smem)),
                 "l"(src), "r"(bytes), "r"(shmemg_smem_u32(bar))
                 : "memory");
}

template <typename T, typename V, int OP>
__global__ void __launch_bounds__(RB_THREADS, 1) k_reduce_bulk(Red x, uint8_t *state, uint64_t timeout_ns) {
    extern __shared__ __align__(128) uint8_t rb[];
    __shared__ __align__(8) uint64_t bars[RB_MAX_STAGES];
    constexpr int NL = sizeof(V) / sizeof(T);
    const int P = x.size;
    const int pe0 = x.start + blockIdx.y * x.gstride;
    const uint32_t C = x.rb_chunk, S = x.rb_stages, ncol = C / 16, nparts = RB_THREADS / ncol;
    const uint64_t SB = (uint64_t)P * C;  // stage bytes
    const uint32_t col = threadIdx.x % ncol, part = threadIdx.x / ncol, lane = threadIdx.x & 31;
    const uint64_t bytes = x.nvec * sizeof(V);  // per member
    const uint64_t nchunks = (bytes + C - 1) / C;
    if (nchunks <= blockIdx.x) return;  // (uniform over the CTA)
    const uint64_t count = (nchunks - blockIdx.x + gridDim.x - 1) / gridDim.x;
    V *partial = (V *)(rb + RB_RING);
    auto chunk_bytes = [&](uint64_t c) { return (uint32_t)(bytes - c * C < C ? bytes - c * C : C); };
    auto issue = [&](uint64_t j) {  // warp 0: chunk j's member loads into stage j % S
        const uint64_t c = blockIdx.x + j * gridDim.x;
        const uint32_t b = chunk_bytes(c), s = (uint32_t)(j % S);
        uint8_t *stage = rb + s * SB;
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(shmemg_smem_u32(&bars[s])),
                         "r"(b * (uint32_t)P)
                         : "memory");
        __syncwarp();
        for (int r = (int)lane; r < P; r += 32)
            rb_load(stage + (uint64_t)r * C, x.heap + (uint64_t)(pe0 + r * x.stride) * x.H + x.src_off + c * C, b,
                    &bars[s]);
    };
    auto comb = [&](V &a, const V &b) {
#pragma unroll
        for (int l = 0; l < NL; l++)
            reinterpret_cast<T *>(&a)[l] = shmemg_comb<T>(reinterpret_cast<T *>(&a)[l], reinterpret_cast<const T *>(&b)[l], OP);
    };
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < S; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shmemg_smem_u32(&bars[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x < 32)
        for (uint64_t j = 0; j < count && j < S; j++) issue(j);
    for (uint64_t j = 0; j < count; j++) {
        const uint32_t s = (uint32_t)(j % S);
        const bool ok = shmemg_mbar_wait(&bars[s], (uint32_t)((j / S) & 1), timeout_ns);
        const uint64_t c = blockIdx.x + j * gridDim.x;
        const uint32_t nc = chunk_bytes(c) / 16;
        V *pb = partial + (j & 1) * RB_THREADS;  // (double-buffered: chunk j + 2 writes after barrier j + 1)
        if (ok && col < nc) {
            const uint8_t *stage = rb + s * SB + (uint64_t)col * 16;
            V acc = *(const V *)(stage + (uint64_t)part * C);
            int r = (int)(part + nparts);
            for (; r + 3 * (int)nparts < P; r += 4 * (int)nparts) {
                V v[4];
#pragma unroll
                for (int u = 0; u < 4; u++) v[u] = *(const V *)(stage + (uint64_t)(r + u * (int)nparts) * C);
#pragma unroll
                for (int u = 0; u < 4; u++) comb(acc, v[u]);
            }
            for (; r < P; r += (int)nparts) comb(acc, *(const V *)(stage + (uint64_t)r * C));
            pb[threadIdx.x] = acc;
        }
        if (__syncthreads_or(!ok)) {  // a stage never landed: every thread stops here
            if (threadIdx.x == 0) {
                // no load of the ring may still be writing shared memory when the CTA exits
                const bool drained = shmemg_bulk_drain_loads(bars, S, j, count, timeout_ns);
                int *st = (int *)(state + SHMEMG_STATUS_OFF);
                if (atomicCAS(st, 0, SHMEMG_ERR_TIMEOUT) == 0)
                    *(volatile int64_t *)(state + SHMEMG_STATUS_OFF + 8) = drained ? -3 : -4;
            }
            break;
        }
        // every thread has read stage s: warp 0 refills it while the groups store chunk j
        if (threadIdx.x < 32 && j + S < count) issue(j + S);
        if (col < nc) {
            V acc = pb[col];
            for (uint32_t q = 1; q < nparts; q++) comb(acc, pb[q * ncol + col]);
            const uint64_t doff = x.dst_off + c * C + (uint64_t)col * 16;
            for (int r = (int)part; r < P; r += (int)nparts)
                *(V *)(x.heap + (uint64_t)(pe0 + r * x.stride) * x.H + doff) = acc;
        }
    }
}

// ------------------------------------------------------------------ single-thread ops
template <typename T>
__global__ void k_amo(T *addr, int kind, T v, T cond, T *fetched) {
    T old;
    if (kind == SHMEMG_OP_FETCH_ADD) old = atomicAdd(addr, v);
    else if (kind == SHMEMG_OP_COMPARE_SWAP) old = atomicCAS(addr, cond, v);
    else old = atomicXor(addr, v);
    if (fetched) *fetched = old;
}

__global__ void k_wait(shmemg_device_ctx_t c, const uint64_t *sig, int cmp, uint64_t val) {
    shmemg_d_signal_wait_until(c, sig, cmp, val, -1);
}

// ------------------------------------------------------------------ launch helpers
static int vec_width(uint64_t m) {
    return (m & 15) == 0 ? 16 : (m & 7) == 0 ? 8 : (m & 3) == 0 ? 4 : (m & 1) == 0 ? 2 : 1;
}

// Destination members per item of a replicating transfer (broadcast, fcollect): a
// launch with fewer segment chunks than resident CTAs splits each chunk's member stores
// over several items (each reads the chunk -- from L2 after the first), so the stores
// spread over the GPU instead of one CTA writing every member's copy.
static int member_groups(const Xfer &x, uint64_t items, uint64_t cap, int ngroups) {
    if ((x.kind != X_BCAST && x.kind != X_FCOLLECT) || items == 0) return 1;
    if (ngroups > 1) cap = cap / (uint64_t)ngroups > 0 ? cap / (uint64_t)ngroups : 1;
    if (items >= cap) return 1;
    const uint64_t g = (cap + items - 1) / items;
    return (int)(g < (uint64_t)x.size ? g : (uint64_t)x.size);
}

template <typename V>
static int launch_xfer_v(Xfer x, int ngroups, cudaStream_t s, uint64_t *sig, uint64_t val, int op, uint32_t *done) {
    x.seg_vec /= sizeof(V);
    x.chunk_vec = (uint64_t)XFER_THREADS * XFER_U;
    x.chunks_per_seg = (x.seg_vec + x.chunk_vec - 1) / x.chunk_vec;
    if (x.chunks_per_seg == 0) x.chunks_per_seg = 1;
    uint64_t nseg = x.kind == X_A2A ? (uint64_t)x.size * x.size : x.kind == X_FCOLLECT ? (uint64_t)x.size : 1;
    x.nitems = x.seg_vec ? nseg * x.chunks_per_seg : 0;
    if (x.nitems == 0 && !sig) return SHMEMG_SUCCESS;
    const void *kfn = sig ? (const void *)k_put_signal<V> : (const void *)k_xfer<V>;
    const uint64_t cap = (uint64_t)ctas_for(kfn, XFER_THREADS, 0);
    x.mgroups = member_groups(x, x.nitems, cap, ngroups);
    x.nitems *= (uint64_t)x.mgroups;
    const uint64_t gx = balanced_grid(x.nitems, cap, ngroups);
    dim3 grid((unsigned)gx, (unsigned)ngroups);
    if (sig) k_put_signal<V><<<grid, XFER_THREADS, 0, s>>>(x, sig, val, op, done);
    else k_xfer<V><<<grid, XFER_THREADS, 0, s>>>(x);
    return cuda_rc(cudaGetLastError());
}

static bool bulk_enabled() {
    static int on = -1;
    if (on < 0) {
        const char *e = getenv("SHMEMG_BULK");
        on = (e && *e == '0') ? 0 : 1;
        if (on && cudaFuncSetAttribute((const void *)k_xfer_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       XB_SMEM) != cudaSuccess) {
            cudaGetLastError();
            on = 0;
        }
    }
    return on == 1;
}

// segments of >= one chunk with 16-byte aligned addresses and lengths go to the bulk engine
static int launch_xfer_bulk(Xfer x, int ngroups, cudaStream_t s) {
    x.chunks_per_seg = (x.seg_vec + XB_CHUNK - 1) / XB_CHUNK;
    const uint64_t nseg = x.kind == X_A2A ? (uint64_t)x.size * x.size : x.kind == X_FCOLLECT ? (uint64_t)x.size : 1;
    x.nitems = nseg * x.chunks_per_seg;
    const uint64_t cap = (uint64_t)ctas_for((const void *)k_xfer_bulk, 32, XB_SMEM);
    x.mgroups = member_groups(x, x.nitems, cap, ngroups);
    x.nitems *= (uint64_t)x.mgroups;
    dim3 grid((unsigned)balanced_grid(x.nitems, cap, ngroups), (unsigned)ngroups);
    k_xfer_bulk<<<grid, 32, XB_SMEM, s>>>(x, st().base, st().timeout_ns);
    return cuda_rc(cudaGetLastError());
}

// x.seg_vec carries the segment length in BYTES on entry
static int launch_xfer(Xfer x, int ngroups, uint64_t align_bits, cudaStream_t s, uint64_t *sig = nullptr,
                       uint64_t val = 0, int op = 0, uint32_t *done = nullptr) {
    // (alltoall's many smaller segments measured faster on the vector path)
    if (!sig && x.kind != X_A2A && ((align_bits | x.seg_vec) & 15) == 0 && x.seg_vec >= XB_CHUNK && bulk_enabled())
        return launch_xfer_bulk(x, ngroups, s);
    switch (vec_width(align_bits | x.seg_vec)) {
    case 16: return launch_xfer_v<uint4>(x, ngroups, s, sig, val, op, done);
    case 8: return launch_xfer_v<uint2>(x, ngroups, s, sig, val, op, done);
    case 4: return launch_xfer_v<uint32_t>(x, ngroups, s, sig, val, op, done);
    case 2: return launch_xfer_v<uint16_t>(x, ngroups, s, sig, val, op, done);
    default: return launch_xfer_v<uint8_t>(x, ngroups, s, sig, val, op, done);
    }
}

static Xfer xfer_base() {
    Xfer x;
    memset(&x, 0, sizeof(x));
    x.heap = st().heap;
    x.H = st().H;
    x.stride = 1;
    x.mgroups = 1;
    return x;
}

static int rma(void *dst, const void *src, uint64_t n, int dst_pe, int src_pe, void *stream) {
    if (int rc = check_init()) return rc;
    if (check_pe(dst_pe) || check_pe(src_pe)) return SHMEMG_ERR_INVALID_ARG;
    uint64_t doff, soff;
    if (sym_offset(dst, n, &doff) || sym_offset(src, n, &soff)) return SHMEMG_ERR_NOT_SYMMETRIC;
    if (n == 0) return SHMEMG_SUCCESS;
    Xfer x = xfer_base();
    x.kind = X_COPY;
    x.size = 1;
    x.dst_pe = dst_pe;
    x.src_pe = src_pe;
    x.dst_off = doff;
    x.src_off = soff;
    x.seg_vec = n;
    return launch_xfer(x, 1, doff | soff, to_stream(stream));
}

// bytes per member from which integer reductions take the bulk ring (SHMEMG_RED_BULK_MIN
// overrides; a value above any partition turns the ring off)
static uint64_t red_bulk_min() {
    static uint64_t v = [] {
        const char *e = getenv("SHMEMG_RED_BULK_MIN");
        return (e && *e) ? (uint64_t)strtoull(e, nullptr, 10) : (uint64_t)(128u << 10);
    }();
    return v;
}

// ring shape for a P-member team: 1 KiB per member per chunk, three stages; only teams of
// 48..64 members (the measured range where the ring beats the register form; see
// k_reduce_bulk)
static bool rb_shape(int P, uint32_t *chunk, uint32_t *stages) {
    *chunk = 1024;
    *stages = 3;
    return P >= 48 && P <= 64;
}

// the ring's shared memory granted to kernel `k` (once per instantiation)
static bool red_bulk_ready(const void *k) {
    static std::mutex mu;
    static std::unordered_map<const void *, bool> ok;
    std::lock_guard<std::mutex> lk(mu);
    auto it = ok.find(k);
    if (it != ok.end()) return it->second;
    const bool g = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, RB_SMEM) == cudaSuccess;
    if (!g) cudaGetLastError();
    ok[k] = g;
    return g;
}

template <typename V, typename T, int OP>
static int launch_red_v(Red r, int ngroups, cudaStream_t s) {
    r.nvec /= (sizeof(V) / sizeof(T));
    r.chunk_vec = (uint64_t)RED_THREADS * RED_U;
    r.nitems = (r.nvec + r.chunk_vec - 1) / r.chunk_vec;
    if (r.nitems == 0) return SHMEMG_SUCCESS;
    if constexpr (std::is_integral<T>::value && sizeof(V) == 16) {
        // integer teams of 48..64 members with 128 KiB .. 16 MiB per member: the bulk ring
        // (above 16 MiB both forms run at the HBM rate and the register form is the steadier)
        if ((r.H & 15) == 0 && r.nvec * sizeof(V) >= red_bulk_min() && r.nvec * sizeof(V) <= RB_MAX_BYTES &&
            rb_shape(r.size, &r.rb_chunk, &r.rb_stages) && red_bulk_ready((const void *)k_reduce_bulk<T, V, OP>)) {
            const uint64_t C = r.rb_chunk, nchunks = (r.nvec * sizeof(V) + C - 1) / C;
            const uint64_t cap = (uint64_t)ctas_for((const void *)k_reduce_bulk<T, V, OP>, RB_THREADS, RB_SMEM);
            dim3 grid((unsigned)balanced_grid(nchunks, cap, ngroups), (unsigned)ngroups);
            k_reduce_bulk<T, V, OP><<<grid, RB_THREADS, RB_SMEM, s>>>(r, st().base, st().timeout_ns);
            return cuda_rc(cudaGetLastError());
        }
        // integer teams with too few vectors to fill the GPU one thread each: several
        // threads per vector (k_reduce_split)
        const int G = r.size >= 32 ? 8 : r.size >= 8 ? 4 : 1;
        const void *kf = G == 8 ? (const void *)k_reduce_split<T, V, OP, 8> : (const void *)k_reduce_split<T, V, OP, 4>;
        if (G > 1) {
            const uint64_t cap = (uint64_t)ctas_for(kf, RED_THREADS, 0);
            const uint64_t ctas = (r.nvec * G + RED_THREADS - 1) / RED_THREADS;
            // (measured: 4-5x faster up to 64 Ki vectors per member; once the one-per-thread
            // form has a few hundred items its coalesced member loads win)
            if (r.nitems * (uint64_t)ngroups * 8 < cap) {
                dim3 grid((unsigned)balanced_grid(ctas, cap, ngroups), (unsigned)ngroups);
                if (G == 8) k_reduce_split<T, V, OP, 8><<<grid, RED_THREADS, 0, s>>>(r);
                else k_reduce_split<T, V, OP, 4><<<grid, RED_THREADS, 0, s>>>(r);
                return cuda_rc(cudaGetLastError());
            }
        }
    }
    const void *kfn = (const void *)k_reduce<T, V, OP>;
    const uint64_t cap = (uint64_t)ctas_for(kfn, RED_THREADS, 0);
    if (r.nitems * (uint64_t)ngroups < cap) {  // too few items for the resident CTAs: one vector per thread
        r.chunk_vec = RED_THREADS;
        r.nitems = (r.nvec + r.chunk_vec - 1) / r.chunk_vec;
    }
    dim3 grid((unsigned)balanced_grid(r.nitems, cap, ngroups), (unsigned)ngroups);
    k_reduce<T, V, OP><<<grid, RED_THREADS, 0, s>>>(r);
    return cuda_rc(cudaGetLastError());
}

template <typename T, typename V16, int OP>
static int launch_red(Red r, int ngroups, bool vec_ok, cudaStream_t s) {
    return vec_ok ? launch_red_v<V16, T, OP>(r, ngroups, s) : launch_red_v<T, T, OP>(r, ngroups, s);
}

}  // namespace shmemg

using namespace shmemg;

// ================================================================== C ABI
extern "C" {

int shmemg_putmem(void *dst, const void *src, uint64_t n, int pe, int issuer, void *stream) {
    return rma(dst, src, n, pe, issuer, stream);
}
int shmemg_putmem_nbi(void *dst, const void *src, uint64_t n, int pe, int issuer, void *stream) {
    return rma(dst, src, n, pe, issuer, stream);
}
int shmemg_getmem(void *dst, const void *src, uint64_t n, int pe, int issuer, void *stream) {
    return rma(dst, src, n, issuer, pe, stream);
}
int shmemg_getmem_nbi(void *dst, const void *src, uint64_t n, int pe, int issuer, void *stream) {
    return rma(dst, src, n, issuer, pe, stream);
}

}  // extern "C"

template <typename T>
static int amo(T *target, int kind, T v, T cond, int pe, T *fetched, void *stream) {
    if (int rc = check_init()) return rc;
    if (check_pe(pe)) return SHMEMG_ERR_INVALID_ARG;
    uint64_t off;
    if (sym_offset(target, sizeof(T), &off)) return SHMEMG_ERR_NOT_SYMMETRIC;
    if (off % sizeof(T)) return SHMEMG_ERR_INVALID_ARG;
    T *addr = (T *)(st().heap + (uint64_t)pe * st().H + off);
    k_amo<T><<<1, 1, 0, to_stream(stream)>>>(addr, kind, v, cond, fetched);
    return cuda_rc(cudaGetLastError());
}

extern "C" {

int shmemg_int64_atomic_fetch_add(int64_t *t, int64_t v, int pe, int64_t *f, void *s) {
    return amo<unsigned long long>((unsigned long long *)t, SHMEMG_OP_FETCH_ADD, (unsigned long long)v, 0ull, pe,
                                   (unsigned long long *)f, s);
}
int shmemg_int64_atomic_compare_swap(int64_t *t, int64_t c, int64_t v, int pe, int64_t *f, void *s) {
    return amo<unsigned long long>((unsigned long long *)t, SHMEMG_OP_COMPARE_SWAP, (unsigned long long)v,
                                   (unsigned long long)c, pe, (unsigned long long *)f, s);
}
int shmemg_int64_atomic_fetch_xor(int64_t *t, int64_t v, int pe, int64_t *f, void *s) {
    return amo<unsigned long long>((unsigned long long *)t, SHMEMG_OP_FETCH_XOR, (unsigned long long)v, 0ull, pe,
                                   (unsigned long long *)f, s);
}
int shmemg_int32_atomic_fetch_add(int32_t *t, int32_t v, int pe, int32_t *f, void *s) {
    return amo<int>((int *)t, SHMEMG_OP_FETCH_ADD, v, 0, pe, (int *)f, s);
}
int shmemg_int32_atomic_compare_swap(int32_t *t, int32_t c, int32_t v, int pe, int32_t *f, void *s) {
    return amo<int>((int *)t, SHMEMG_OP_COMPARE_SWAP, v, c, pe, (int *)f, s);
}
int shmemg_int32_atomic_fetch_xor(int32_t *t, int32_t v, int pe, int32_t *f, void *s) {
    return amo<int>((int *)t, SHMEMG_OP_FETCH_XOR, v, 0, pe, (int *)f, s);
}

int shmemg_putmem_signal(void *dst, const void *src, uint64_t n, uint64_t *sig, uint64_t sigval, int sig_op,
                         int pe, int issuer, void *stream) {
    if (int rc = check_init()) return rc;
    if (check_pe(pe) || check_pe(issuer)) return SHMEMG_ERR_INVALID_ARG;
    if (sig_op != SHMEMG_SIGNAL_SET && sig_op != SHMEMG_SIGNAL_ADD) return SHMEMG_ERR_INVALID_ARG;
    uint64_t doff, soff, goff;
    if (sym_offset(dst, n, &doff) || sym_offset(src, n, &soff) || sym_offset(sig, 8, &goff))
        return SHMEMG_ERR_NOT_SYMMETRIC;
    if (goff & 7) return SHMEMG_ERR_INVALID_ARG;
    State &S = st();
    Xfer x = xfer_base();
    x.kind = X_COPY;
    x.size = 1;
    x.dst_pe = pe;
    x.src_pe = issuer;
    x.dst_off = doff;
    x.src_off = soff;
    x.seg_vec = n;
    uint32_t *done = (uint32_t *)(S.base + SHMEMG_SCRATCH_OFF + SCR_SIGNAL_DONE) +
                     (S.call_seq++ % SCR_SIGNAL_DONE_SLOTS);
    uint64_t *sig_addr = (uint64_t *)(S.heap + (uint64_t)pe * S.H + goff);
    return launch_xfer(x, 1, doff | soff, to_stream(stream), sig_addr, sigval, sig_op, done);
}

int shmemg_signal_wait_until(uint64_t *sig, int pe, int cmp, uint64_t value, void *stream) {
    if (int rc = check_init()) return rc;
    if (check_pe(pe) || cmp < SHMEMG_CMP_EQ || cmp > SHMEMG_CMP_LE) return SHMEMG_ERR_INVALID_ARG;
    uint64_t off;
    if (sym_offset(sig, 8, &off) || (off & 7)) return SHMEMG_ERR_NOT_SYMMETRIC;
    k_wait<<<1, 1, 0, to_stream(stream)>>>(device_ctx(), (const uint64_t *)(st().heap + (uint64_t)pe * st().H + off),
                                          cmp, value);
    return cuda_rc(cudaGetLastError());
}

// --------------------------------------------------------------- collectives
static int coll_prep(shmemg_team_t team, HostTeam *t) {
    if (int rc = check_init()) return rc;
    if (team_get(team, t)) return SHMEMG_ERR_INVALID_ARG;
    return SHMEMG_SUCCESS;
}

static Xfer team_xfer(const HostTeam &t, int kind) {
    Xfer x = xfer_base();
    x.kind = kind;
    x.start = t.start;
    x.stride = t.stride;
    x.size = t.size;
    x.gstride = t.gstride;
    return x;
}

int shmemg_broadcastmem(shmemg_team_t team, void *dst, const void *src, uint64_t n, int root, void *stream) {
    HostTeam t;
    if (int rc = coll_prep(team, &t)) return rc;
    if (root < 0 || root >= t.size) return SHMEMG_ERR_INVALID_ARG;
    uint64_t doff, soff;
    if (sym_offset(dst, n, &doff) || sym_offset(src, n, &soff)) return SHMEMG_ERR_NOT_SYMMETRIC;
    if (n == 0) return SHMEMG_SUCCESS;
    Xfer x = team_xfer(t, X_BCAST);
    x.root = root;
    x.dst_off = doff;
    x.src_off = soff;
    x.seg_vec = n;
    return launch_xfer(x, t.ngroups, doff | soff, to_stream(stream));
}

int shmemg_fcollectmem(shmemg_team_t team, void *dst, const void *src, uint64_t n, void *stream) {
    HostTeam t;
    if (int rc = coll_prep(team, &t)) return rc;
    uint64_t doff, soff;
    if (sym_offset(dst, n * (uint64_t)t.size, &doff) || sym_offset(src, n, &soff)) return SHMEMG_ERR_NOT_SYMMETRIC;
    if (n == 0) return SHMEMG_SUCCESS;
    Xfer x = team_xfer(t, X_FCOLLECT);
    x.dst_off = doff;
    x.src_off = soff;
    x.seg_vec = n;
    return launch_xfer(x, t.ngroups, doff | soff, to_stream(stream));
}

int shmemg_alltoallmem(shmemg_team_t team, void *dst, const void *src, uint64_t n, void *stream) {
    HostTeam t;
    if (int rc = coll_prep(team, &t)) return rc;
    uint64_t doff, soff;
    uint64_t tot = n * (uint64_t)t.size;
    if (sym_offset(dst, tot, &doff) || sym_offset(src, tot, &soff)) return SHMEMG_ERR_NOT_SYMMETRIC;
    if (n == 0) return SHMEMG_SUCCESS;
    Xfer x = team_xfer(t, X_A2A);
    x.dst_off = doff;
    x.src_off = soff;
    x.seg_vec = n;
    return launch_xfer(x, t.ngroups, doff | soff, to_stream(stream));
}

int shmemg_reduce(shmemg_team_t team, void *dst, const void *src, uint64_t nelems, int dtype, int op,
                  void *stream) {
    HostTeam t;
    if (int rc = coll_prep(team, &t)) return rc;
    if (op != SHMEMG_SUM && op != SHMEMG_MAX && op != SHMEMG_MIN) return SHMEMG_ERR_INVALID_ARG;
    uint64_t es = dtype == SHMEMG_INT64 ? 8 : (dtype == SHMEMG_INT32 || dtype == SHMEMG_FLOAT) ? 4 : 0;
    if (!es) return SHMEMG_ERR_INVALID_ARG;
    uint64_t doff, soff;
    if (sym_offset(dst, nelems * es, &doff) || sym_offset(src, nelems * es, &soff)) return SHMEMG_ERR_NOT_SYMMETRIC;
    if (doff % es || soff % es) return SHMEMG_ERR_INVALID_ARG;
    // dst == src (in place) is fine: each element is read by its owner before written;
    // partial overlaps are undefined
    if (doff != soff && doff < soff + nelems * es && soff < doff + nelems * es) return SHMEMG_ERR_INVALID_ARG;
    if (nelems == 0) return SHMEMG_SUCCESS;
    Red r;
    memset(&r, 0, sizeof(r));
    r.heap = st().heap;
    r.H = st().H;
    r.start = t.start;
    r.stride = t.stride;
    r.size = t.size;
    r.gstride = t.gstride;
    r.dst_off = doff;
    r.src_off = soff;
    r.nvec = nelems;
    bool v16 = ((doff | soff | (nelems * es)) & 15) == 0;
    cudaStream_t s = to_stream(stream);
    int g = t.ngroups;
#define SHMEMG_RED(T, V) \
    (op == SHMEMG_SUM ? launch_red<T, V, SHMEMG_SUM>(r, g, v16, s) \
     : op == SHMEMG_MAX ? launch_red<T, V, SHMEMG_MAX>(r, g, v16, s) : launch_red<T, V, SHMEMG_MIN>(r, g, v16, s))
    if (dtype == SHMEMG_INT32) return SHMEMG_RED(int32_t, int4);
    if (dtype == SHMEMG_INT64) return SHMEMG_RED(int64_t, longlong2);
    return SHMEMG_RED(float, float4);
#undef SHMEMG_RED
}

#define SHMEMG_NAMED_REDUCE(name, T, DT, OP)                                                          \
    int shmemg_##name##_reduce(shmemg_team_t team, T *dst, const T *src, uint64_t n, void *stream) { \
        return shmemg_reduce(team, dst, src, n, DT, OP, stream);                                      \
    }
SHMEMG_NAMED_REDUCE(int32_sum, int32_t, SHMEMG_INT32, SHMEMG_SUM)
SHMEMG_NAMED_REDUCE(int32_max, int32_t, SHMEMG_INT32, SHMEMG_MAX)
SHMEMG_NAMED_REDUCE(int32_min, int32_t, SHMEMG_INT32, SHMEMG_MIN)
SHMEMG_NAMED_REDUCE(int64_sum, int64_t, SHMEMG_INT64, SHMEMG_SUM)
SHMEMG_NAMED_REDUCE(int64_max, int64_t, SHMEMG_INT64, SHMEMG_MAX)
SHMEMG_NAMED_REDUCE(int64_min, int64_t, SHMEMG_INT64, SHMEMG_MIN)
SHMEMG_NAMED_REDUCE(float_sum, float, SHMEMG_FLOAT, SHMEMG_SUM)
SHMEMG_NAMED_REDUCE(float_max, float, SHMEMG_FLOAT, SHMEMG_MAX)
SHMEMG_NAMED_REDUCE(float_min, float, SHMEMG_FLOAT, SHMEMG_MIN)

// --------------------------------------------------------------- host script runner
int shmemg_run_script_host(const shmemg_op_t *ops, int64_t nops, int64_t *fetched, void *stream) {
    if (int rc = check_init()) return rc;
    if (nops < 0 || (nops && !ops)) return SHMEMG_ERR_INVALID_ARG;
    State &S = st();
    for (int64_t i = 0; i < nops; i++) {
        const shmemg_op_t &o = ops[i];
        uint8_t *dst = S.heap + o.dst, *src = S.heap + o.src;
        int rc = SHMEMG_SUCCESS;
        // a host-issued op has no thread scope: the warp-scope flag selects the same op
        if ((o.kind & ~SHMEMG_OP_KIND_MASK) & ~SHMEMG_OP_WARP) return SHMEMG_ERR_INVALID_ARG;
        switch (o.kind & SHMEMG_OP_KIND_MASK) {
        case SHMEMG_OP_PUT: rc = shmemg_putmem(dst, src, o.n, o.pe, o.issuer, stream); break;
        case SHMEMG_OP_PUT_NBI: rc = shmemg_putmem_nbi(dst, src, o.n, o.pe, o.issuer, stream); break;
        case SHMEMG_OP_GET: rc = shmemg_getmem(dst, src, o.n, o.pe, o.issuer, stream); break;
        case SHMEMG_OP_GET_NBI: rc = shmemg_getmem_nbi(dst, src, o.n, o.pe, o.issuer, stream); break;
        case SHMEMG_OP_FETCH_ADD:
        case SHMEMG_OP_COMPARE_SWAP:
        case SHMEMG_OP_FETCH_XOR:
            if (o.dtype == SHMEMG_INT64) {
                if (o.kind == SHMEMG_OP_FETCH_ADD)
                    rc = shmemg_int64_atomic_fetch_add((int64_t *)dst, o.operand, o.pe, fetched ? fetched + i : nullptr, stream);
                else if (o.kind == SHMEMG_OP_COMPARE_SWAP)
                    rc = shmemg_int64_atomic_compare_swap((int64_t *)dst, o.cond, o.operand, o.pe,
                                                          fetched ? fetched + i : nullptr, stream);
                else
                    rc = shmemg_int64_atomic_fetch_xor((int64_t *)dst, o.operand, o.pe, fetched ? fetched + i : nullptr, stream);
            } else {
                rc = SHMEMG_ERR_UNSUPPORTED;  // int32 AMOs are host calls of their own
            }
            break;
        case SHMEMG_OP_PUT_SIGNAL:
            rc = shmemg_putmem_signal(dst, src, o.n, (uint64_t *)(S.heap + o.aux), (uint64_t)o.operand, o.sub, o.pe,
                                      o.issuer, stream);
            break;
        case SHMEMG_OP_WAIT_UNTIL:
            rc = shmemg_signal_wait_until((uint64_t *)dst, o.issuer, o.sub, (uint64_t)o.operand, stream);
            break;
        case SHMEMG_OP_BARRIER_ALL: rc = shmemg_barrier_all(stream); break;
        case SHMEMG_OP_QUIET: rc = shmemg_quiet(stream); break;
        case SHMEMG_OP_FENCE: rc = shmemg_fence(stream); break;
        case SHMEMG_OP_TEAM_SYNC: rc = shmemg_team_sync(o.team, stream); break;
        case SHMEMG_OP_BROADCAST: rc = shmemg_broadcastmem(o.team, dst, src, o.n, o.pe, stream); break;
        case SHMEMG_OP_FCOLLECT: rc = shmemg_fcollectmem(o.team, dst, src, o.n, stream); break;
        case SHMEMG_OP_ALLTOALL: rc = shmemg_alltoallmem(o.team, dst, src, o.n, stream); break;
        case SHMEMG_OP_REDUCE: rc = shmemg_reduce(o.team, dst, src, o.n, o.dtype, o.sub, stream); break;
        default: rc = SHMEMG_ERR_INVALID_ARG;
        }
        if (rc) return rc;
    }
    return SHMEMG_SUCCESS;
}

}  // extern "C"
