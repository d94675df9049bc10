// Device-initiated execution of a scripted operation list (paper Sec. 6.3,
// device-initiated path; Fig. 6b: put -> fence -> quiet issued by GPU threads).
//
// One cooperative launch holds every PE (a CTA, or a cluster of CTAs in pe_mode
// CLUSTER).  Every PE walks the whole list; it issues, in list order, the RMA/AMO/signal
// ops whose issuer it is, and its share of every collective of a team it belongs to.
// Blocking RMA ends with a PE barrier (local completion, and later ops of the PE see
// it); collectives and barriers quiet and synchronise their team on entry and exit.
#include <cuda_runtime.h>

#include <cstdlib>

#include "internal.h"

namespace shmemg {

constexpr int INTERP_THREADS = 512;
constexpr int OP_BATCH = 64;  // op records staged in shared memory at a time

// Large aligned puts and gets (>= SHMEMG_BULK_MIN) run on the bulk (TMA) engine when the
// launch provides its shared-memory ring (use_bulk): thread 0 of each CTA of the PE
// streams every ncta-th chunk.
__device__ __forceinline__ void pe_copy(const shmemg_device_ctx_t &c, shmemg_group g, uint8_t *d, const uint8_t *s,
                                        uint64_t n, int use_bulk, uint8_t *ring, uint64_t *bars) {
    if (use_bulk && n >= SHMEMG_BULK_MIN && (((uint64_t)d | (uint64_t)s | n) & 15) == 0) {
        // the split follows the hardware cluster shape: a launch without clusters (each
        // CTA its own cluster of one) still copies every chunk
        const bool cl = c.pe_mode == SHMEMG_PE_MODE_CLUSTER;
        if (threadIdx.x == 0)
            shmemg_d_bulk_copy_thread(c, d, s, n, cl ? shmemg_d_cluster_ctarank() : 0u,
                                      cl ? shmemg_d_cluster_nctarank() : 1u, ring, bars);
    } else {
        shmemg_d_copy_group(g, d, s, n);
    }
}

// ---------------------------------------------------------------- explicit contexts
// Explicit device contexts (Sec. 6.2: contexts as independent ordering and completion
// domains, an optional resource-limited feature beside the default device context).
// Context k (1..SHMEMG_DEVICE_CTX_COUNT-1) of a PE is served by one thread of the PE's
// leader CTA, thread 32*k, with a ring of CTX_STAGES shared-memory stages, one mbarrier
// per stage and the thread's own bulk-group queue: its put_nbi / get_nbi are queued and
// moved chunk by chunk with TMA bulk copies (global -> shared -> global) that run while
// the PE goes on with later ops -- the thread advances them without blocking at every op
// boundary -- and only quiet / fence on that context (or on all of them) waits for them.
// Context 0, the default context, completes its non-blocking ops as it issues them.
constexpr int CTX_STAGES = 2;
constexpr uint32_t CTX_CHUNK = 12u << 10;
constexpr int CTX_QCAP = 8;
constexpr size_t CTX_SMEM = (size_t)(SHMEMG_DEVICE_CTX_COUNT - 1) * CTX_STAGES * CTX_CHUNK;

struct CtxXfer {
    uint64_t dst, src, n;  // generic global addresses, 16-byte multiples
};
// Chunks are numbered across the context's transfers; chunk k uses stage k % CTX_STAGES,
// its load completes phase (k / CTX_STAGES) & 1 of that stage's mbarrier.
struct CtxState {
    CtxXfer q[CTX_QCAP];
    uint32_t head, tail;              // queued transfers; q[head] is being loaded
    uint64_t off;                     // bytes of q[head] whose loads are issued
    uint64_t ld, st;                  // chunks whose loads / stores are issued
    uint64_t st_dst[CTX_STAGES];      // where each stage's chunk goes, and its length
    uint32_t st_len[CTX_STAGES];
    uint64_t bar[CTX_STAGES];
};

__device__ __forceinline__ bool ctx_mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(shmemg_smem_u32(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

// Issues what can be issued now without waiting: stores of chunks whose loads have
// landed, then loads into stages whose previous chunk's store has read them.
__device__ __forceinline__ void ctx_progress(CtxState &x, uint8_t *ring) {
    while (x.st < x.ld) {
        const uint32_t s = (uint32_t)(x.st % CTX_STAGES);
        if (!ctx_mbar_test(&x.bar[s], (uint32_t)((x.st / CTX_STAGES) & 1))) break;
        shmemg_bulk_store((void *)x.st_dst[s], ring + (size_t)s * CTX_CHUNK, x.st_len[s]);
        x.st++;
    }
    while (x.head != x.tail && x.ld < x.st + CTX_STAGES) {
        if (x.ld >= CTX_STAGES) {  // the stage's previous chunk: its store must have read it
            const uint32_t newer = (uint32_t)(x.st - (x.ld - CTX_STAGES) - 1);
            if (newer == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            else asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");  // CTX_STAGES == 2: newer <= 1
        }
        const CtxXfer &t = x.q[x.head % CTX_QCAP];
        const uint32_t len = (uint32_t)(t.n - x.off < CTX_CHUNK ? t.n - x.off : CTX_CHUNK);
        const uint32_t s = (uint32_t)(x.ld % CTX_STAGES);
        x.st_dst[s] = t.dst + x.off;
        x.st_len[s] = len;
        shmemg_bulk_load(ring + (size_t)s * CTX_CHUNK, (const void *)(t.src + x.off), len, &x.bar[s]);
        x.ld++;
        x.off += len;
        if (x.off == t.n) {
            x.head++;
            x.off = 0;
        }
    }
}

// Completes every transfer of the context (bounded waits; a load that never lands is
// recorded as a timeout) and makes its writes visible to generic loads.
__device__ __forceinline__ void ctx_drain(const shmemg_device_ctx_t &c, CtxState &x, uint8_t *ring) {
    for (;;) {
        ctx_progress(x, ring);
        if (x.head == x.tail && x.st == x.ld) break;
        if (x.st < x.ld) {
            const uint32_t s = (uint32_t)(x.st % CTX_STAGES);
            if (!shmemg_mbar_wait(&x.bar[s], (uint32_t)((x.st / CTX_STAGES) & 1), c.timeout_ns)) {
                // The other loads in flight land (bounded) before giving up.  The state
                // stays as it is: a stage is reloaded only after its chunk has been
                // stored, so a load that lands late overwrites nothing in use, and the
                // script's final drain waits for it again.
                bool drained = true;
                for (uint64_t k = x.st + 1; k < x.ld; k++)
                    drained = shmemg_mbar_wait(&x.bar[k % CTX_STAGES], (uint32_t)((k / CTX_STAGES) & 1), c.timeout_ns) &&
                              drained;
                shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, drained ? -3 : -4);
                break;
            }
        }
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void ctx_enqueue(const shmemg_device_ctx_t &c, CtxState &x, uint8_t *ring, uint64_t dst,
                                            uint64_t src, uint64_t n) {
    if (x.tail - x.head == CTX_QCAP) ctx_drain(c, x, ring);  // queue full: finish what is queued
    asm volatile("fence.proxy.async.global;" ::: "memory");    // earlier generic writes -> async proxy
    x.q[x.tail % CTX_QCAP] = {dst, src, n};
    x.tail++;
    ctx_progress(x, ring);
}

// A context moves a transfer in the background when the bulk engine is on and the bulk
// copy's 16-byte rule holds; otherwise the op completes at once like the default
// context's (completing earlier than quiet is always allowed).
__device__ __forceinline__ bool ctx_aligned(const shmemg_device_ctx_t &, const void *d, const void *s, uint64_t n,
                                            int use_bulk) {
    return use_bulk && n > 0 && (((uint64_t)d | (uint64_t)s | n) & 15) == 0;
}

// Device-side check of one op (the same rules as the host's argument checks): PEs in
// range, byte ranges inside a partition, AMO alignment, live teams.  Every thread of
// every PE evaluates it on the same record, so the verdict is uniform.
__device__ __forceinline__ bool op_valid(const shmemg_device_ctx_t &c, const shmemg_op_t &o) {
    const uint64_t H = c.pe_stride;
    auto in = [&](uint64_t off, uint64_t n) { return off <= H && n <= H - off; };
    auto pe_ok = [&](int p) { return p >= 0 && p < c.npes; };
    const uint32_t kind = o.kind & SHMEMG_OP_KIND_MASK, flags = o.kind & ~SHMEMG_OP_KIND_MASK;
    if (flags & ~SHMEMG_OP_WARP) return false;
    if (flags) {  // warp scope: RMA, put_signal, barriers and collectives only
        switch (kind) {
        case SHMEMG_OP_PUT: case SHMEMG_OP_GET: case SHMEMG_OP_PUT_NBI: case SHMEMG_OP_GET_NBI:
        case SHMEMG_OP_PUT_SIGNAL: case SHMEMG_OP_BARRIER_ALL: case SHMEMG_OP_TEAM_SYNC: case SHMEMG_OP_BROADCAST:
        case SHMEMG_OP_FCOLLECT: case SHMEMG_OP_ALLTOALL: case SHMEMG_OP_REDUCE:
            break;
        default:
            return false;
        }
    }
    switch (kind) {
    case SHMEMG_OP_PUT: case SHMEMG_OP_GET:
        return pe_ok(o.pe) && pe_ok(o.issuer) && in(o.dst, o.n) && in(o.src, o.n);
    case SHMEMG_OP_PUT_NBI: case SHMEMG_OP_GET_NBI:  // sub: the context
        return pe_ok(o.pe) && pe_ok(o.issuer) && in(o.dst, o.n) && in(o.src, o.n) &&
               o.sub < SHMEMG_DEVICE_CTX_COUNT && (o.sub == 0 || !flags);
    case SHMEMG_OP_FETCH_ADD: case SHMEMG_OP_COMPARE_SWAP: case SHMEMG_OP_FETCH_XOR: {
        const uint64_t es = o.dtype == SHMEMG_INT64 ? 8 : o.dtype == SHMEMG_INT32 ? 4 : 0;
        return es && pe_ok(o.pe) && pe_ok(o.issuer) && in(o.dst, es) && o.dst % es == 0;
    }
    case SHMEMG_OP_PUT_SIGNAL:
        return pe_ok(o.pe) && pe_ok(o.issuer) && in(o.dst, o.n) && in(o.src, o.n) && in(o.aux, 8) && o.aux % 8 == 0 &&
               o.sub <= SHMEMG_SIGNAL_ADD;
    case SHMEMG_OP_WAIT_UNTIL:
        return pe_ok(o.issuer) && in(o.dst, 8) && o.dst % 8 == 0 && o.sub <= SHMEMG_CMP_LE;
    case SHMEMG_OP_QUIET: case SHMEMG_OP_FENCE:  // sub: the context, or SHMEMG_CTX_ALL
        return o.sub < SHMEMG_DEVICE_CTX_COUNT || o.sub == SHMEMG_CTX_ALL;
    case SHMEMG_OP_BARRIER_ALL:
        return true;
    default:
        break;
    }
    if (o.team >= SHMEMG_MAX_TEAMS) return false;
    const shmemg_dteam_t t = *shmemg_d_team(c, o.team);
    if (!t.valid) return false;
    switch (kind) {
    case SHMEMG_OP_TEAM_SYNC: return true;
    case SHMEMG_OP_BROADCAST: return o.pe >= 0 && o.pe < t.size && in(o.dst, o.n) && in(o.src, o.n);
    case SHMEMG_OP_FCOLLECT: return in(o.dst, o.n * (uint64_t)t.size) && in(o.src, o.n);
    case SHMEMG_OP_ALLTOALL: return in(o.dst, o.n * (uint64_t)t.size) && in(o.src, o.n * (uint64_t)t.size);
    case SHMEMG_OP_REDUCE: {
        const uint64_t es = o.dtype == SHMEMG_INT64 ? 8 : (o.dtype == SHMEMG_INT32 || o.dtype == SHMEMG_FLOAT) ? 4 : 0;
        return es && o.sub <= SHMEMG_MIN && in(o.dst, o.n * es) && in(o.src, o.n * es) && o.dst % es == 0 &&
               o.src % es == 0;
    }
    default: return false;
    }
}

// Whether PE `me` does anything for a valid op: RMA, AMO, put-with-signal and waits only
// on their issuing PE, quiet / fence on theirs (or on every PE when issuer < 0); barriers
// and collectives on every PE (membership is decided inside them).
__device__ __forceinline__ bool op_involves(const shmemg_op_t &o, int me) {
    switch (o.kind & SHMEMG_OP_KIND_MASK) {
    case SHMEMG_OP_PUT: case SHMEMG_OP_PUT_NBI: case SHMEMG_OP_GET: case SHMEMG_OP_GET_NBI:
    case SHMEMG_OP_FETCH_ADD: case SHMEMG_OP_COMPARE_SWAP: case SHMEMG_OP_FETCH_XOR:
    case SHMEMG_OP_PUT_SIGNAL: case SHMEMG_OP_WAIT_UNTIL:
        return o.issuer == me;
    case SHMEMG_OP_QUIET: case SHMEMG_OP_FENCE:
        return o.issuer == me || o.issuer < 0;
    default:
        return true;
    }
}

__global__ void __launch_bounds__(INTERP_THREADS) k_interp(shmemg_device_ctx_t c, const shmemg_op_t *ops,
                                                           int64_t nops, int64_t *fetched, int use_bulk) {
    const int me = shmemg_d_my_pe(c);
    const shmemg_group g = shmemg_d_group_pe(c);
    const bool leader = shmemg_d_pe_leader(c);
    __shared__ int s_wrc[2];
    int n_waits = 0;
    extern __shared__ __align__(128) uint8_t s_ring[];
    __shared__ __align__(8) uint64_t s_bars[SHMEMG_BULK_STAGES];
    // the op list is staged through shared memory OP_BATCH records at a time (one
    // coalesced copy per batch instead of a dependent global load per op and thread)
    __shared__ __align__(16) shmemg_op_t s_ops[OP_BATCH];
    // per op of the batch, decoded once by warp 0: 0 = nothing for this PE, 1 = run, 2 = invalid
    __shared__ uint8_t s_act[OP_BATCH];
    // shared-team ops of a CTA-mode heap launched in clusters run inside the cluster: the
    // team barrier is the hardware cluster barrier, small collectives are staged in the
    // bulk ring, which then serves as each CTA's DSMEM window (free between ops: every
    // bulk copy has drained)
    __shared__ shmemg_cluster_state_t s_cs;
    // explicit contexts: served by thread 32*k of the leader CTA (with the bulk ring only)
    __shared__ __align__(16) CtxState s_ctx[SHMEMG_DEVICE_CTX_COUNT - 1];
    const int my_ctx = (use_bulk && shmemg_d_pe_leader_cta(c) && (threadIdx.x & 31) == 0 && threadIdx.x >= 32 &&
                        threadIdx.x < 32 * SHMEMG_DEVICE_CTX_COUNT)
                           ? (int)(threadIdx.x >> 5)
                           : 0;
    uint8_t *ctx_ring = my_ctx ? s_ring + SHMEMG_BULK_SMEM + (size_t)(my_ctx - 1) * CTX_STAGES * CTX_CHUNK : nullptr;
    if (my_ctx) {
        CtxState &x = s_ctx[my_ctx - 1];
        x.head = x.tail = 0;
        x.off = x.ld = x.st = 0;
        for (int k = 0; k < CTX_STAGES; k++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shmemg_smem_u32(&x.bar[k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // (only when the launch really has clusters of cluster_dim CTAs: a launch without
    // them -- a profiler replaying it, say -- runs the shared team on the L2/HBM path and
    // never maps a peer CTA that does not exist)
    const bool dsm = c.pe_mode == SHMEMG_PE_MODE_CTA && c.cluster_dim > 1 &&
                     shmemg_d_cluster_nctarank() == (uint32_t)c.cluster_dim;
    shmemg_cluster_state_t *cs = dsm ? &s_cs : nullptr;
    const uint64_t win_bytes = use_bulk ? SHMEMG_BULK_SMEM : 0;
    if (dsm) shmemg_d_cluster_begin(s_cs);
    auto staged = [&](const shmemg_op_t &o) {
        if (!dsm || o.team != SHMEMG_TEAM_SHARED || (o.kind & SHMEMG_OP_WARP)) return false;
        const uint64_t b = shmemg_d_cluster_stage_bytes(o.kind, o.n, o.dtype, c.cluster_dim);
        return b > 0 && b <= win_bytes;
    };
    // Hardware cluster barriers an op runs on the shared team (a fixed count per op
    // record): a CTA that has failed still passes them for every op it skips, so the
    // CTAs of a cluster always meet at the same barriers (they have no timeout).
    auto cluster_barriers = [&](const shmemg_op_t &o) {
        if (!dsm || o.team != SHMEMG_TEAM_SHARED || (o.kind & SHMEMG_OP_WARP)) return 0;
        switch (o.kind) {
        case SHMEMG_OP_TEAM_SYNC: return 1;
        case SHMEMG_OP_BROADCAST: case SHMEMG_OP_FCOLLECT: case SHMEMG_OP_ALLTOALL: case SHMEMG_OP_REDUCE:
            return staged(o) ? 3 : 2;
        default: return 0;
        }
    };
    bool failed = false;
    for (int64_t base = 0; base < nops && (!failed || dsm); base += OP_BATCH) {
    const int cnt = (int)(nops - base < OP_BATCH ? nops - base : OP_BATCH);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt * 4; q += blockDim.x)
        reinterpret_cast<uint4 *>(s_ops)[q] = __ldcg(reinterpret_cast<const uint4 *>(ops + base) + q);
    __syncthreads();
    // validity and participation once per op and CTA, not once per op and thread: a PE
    // then passes the ops of other PEs in a few instructions
    if (threadIdx.x < 32)
        for (int k = (int)threadIdx.x; k < cnt; k += 32)
            s_act[k] = !op_valid(c, s_ops[k]) ? 2 : op_involves(s_ops[k], me) ? 1 : 0;
    __syncthreads();
    for (int k = 0; k < cnt; k++) {
        const int64_t i = base + k;
        if (my_ctx) ctx_progress(s_ctx[my_ctx - 1], ctx_ring);  // background transfers advance
        const int act = s_act[k];
        if (act == 0 && !failed) continue;
        const shmemg_op_t o = s_ops[k];
        int rc = SHMEMG_SUCCESS;
        if (failed) {  // only in a clustered CTA-mode launch: walk on, through the barriers
            for (int b = cluster_barriers(o); b > 0; b--) shmemg_d_cluster_sync();
            continue;
        }
        if (act == 2) {  // an invalid op ends the script there, recorded with its index
            if (leader) shmemg_d_set_status(c, SHMEMG_ERR_INVALID_ARG, i);
            failed = true;
            if (dsm) continue;
            break;
        }
        // warp scope (SHMEMG_OP_WARP): warp 0 of the PE's leader CTA performs the op with
        // the warp-scope forms; the rest of the PE takes its result afterwards
        const bool warp = (o.kind & SHMEMG_OP_WARP) != 0;
        const bool active =
            !warp || (threadIdx.x < 32 && (c.pe_mode != SHMEMG_PE_MODE_CLUSTER || shmemg_d_cluster_ctarank() == 0));
        const shmemg_group gw = warp ? shmemg_d_group_warp() : g;
        switch (o.kind & SHMEMG_OP_KIND_MASK) {
        case SHMEMG_OP_PUT:
        case SHMEMG_OP_PUT_NBI:
            if (o.issuer == me && o.kind == SHMEMG_OP_PUT_NBI && o.sub != 0 &&
                ctx_aligned(c, shmemg_d_addr(c, o.pe, o.dst), shmemg_d_addr(c, me, o.src), o.n, use_bulk)) {
                if (my_ctx == o.sub)  // queued on its context, moved in the background
                    ctx_enqueue(c, s_ctx[my_ctx - 1], ctx_ring, (uint64_t)shmemg_d_addr(c, o.pe, o.dst),
                                (uint64_t)shmemg_d_addr(c, me, o.src), o.n);
            } else if (o.issuer == me) {
                if (warp) {
                    if (active) shmemg_d_copy_group(gw, shmemg_d_addr(c, o.pe, o.dst), shmemg_d_addr(c, me, o.src), o.n);
                } else {
                    pe_copy(c, g, shmemg_d_addr(c, o.pe, o.dst), shmemg_d_addr(c, me, o.src), o.n, use_bulk, s_ring,
                            s_bars);
                    if (o.kind == SHMEMG_OP_PUT) shmemg_d_pe_sync(c);
                }
            }
            break;
        case SHMEMG_OP_GET:
        case SHMEMG_OP_GET_NBI:
            if (o.issuer == me && o.kind == SHMEMG_OP_GET_NBI && o.sub != 0 &&
                ctx_aligned(c, shmemg_d_addr(c, me, o.dst), shmemg_d_addr(c, o.pe, o.src), o.n, use_bulk)) {
                if (my_ctx == o.sub)
                    ctx_enqueue(c, s_ctx[my_ctx - 1], ctx_ring, (uint64_t)shmemg_d_addr(c, me, o.dst),
                                (uint64_t)shmemg_d_addr(c, o.pe, o.src), o.n);
            } else if (o.issuer == me) {
                if (warp) {
                    if (active) shmemg_d_copy_group(gw, shmemg_d_addr(c, me, o.dst), shmemg_d_addr(c, o.pe, o.src), o.n);
                } else {
                    pe_copy(c, g, shmemg_d_addr(c, me, o.dst), shmemg_d_addr(c, o.pe, o.src), o.n, use_bulk, s_ring,
                            s_bars);
                    if (o.kind == SHMEMG_OP_GET) shmemg_d_pe_sync(c);
                }
            }
            break;
        case SHMEMG_OP_FETCH_ADD:
        case SHMEMG_OP_COMPARE_SWAP:
        case SHMEMG_OP_FETCH_XOR:
            if (o.issuer == me && leader) {
                int64_t old;
                if (o.dtype == SHMEMG_INT64) {
                    int64_t *t = (int64_t *)shmemg_d_addr(c, o.pe, o.dst);
                    if (o.kind == SHMEMG_OP_FETCH_ADD)
                        old = (int64_t)atomicAdd((unsigned long long *)t, (unsigned long long)o.operand);
                    else if (o.kind == SHMEMG_OP_COMPARE_SWAP)
                        old = (int64_t)atomicCAS((unsigned long long *)t, (unsigned long long)o.cond,
                                                 (unsigned long long)o.operand);
                    else
                        old = (int64_t)atomicXor((unsigned long long *)t, (unsigned long long)o.operand);
                } else {
                    int *t = (int *)shmemg_d_addr(c, o.pe, o.dst);
                    if (o.kind == SHMEMG_OP_FETCH_ADD) old = atomicAdd(t, (int)o.operand);
                    else if (o.kind == SHMEMG_OP_COMPARE_SWAP) old = atomicCAS(t, (int)o.cond, (int)o.operand);
                    else old = atomicXor(t, (int)o.operand);
                }
                if (fetched) fetched[i] = old;
            }
            break;
        case SHMEMG_OP_PUT_SIGNAL:
            if (o.issuer == me) {
                if (warp) {
                    if (active)
                        shmemg_d_putmem_signal_warp(c, shmemg_d_addr(c, 0, o.dst), shmemg_d_addr(c, 0, o.src), o.n,
                                                    (uint64_t *)shmemg_d_addr(c, 0, o.aux), (uint64_t)o.operand, o.sub,
                                                    o.pe);
                } else {
                    shmemg_d_copy_group(g, shmemg_d_addr(c, o.pe, o.dst), shmemg_d_addr(c, me, o.src), o.n);
                    shmemg_d_pe_sync(c);
                    if (leader) {
                        shmemg_d_fence_gpu();
                        shmemg_d_signal_op((uint64_t *)shmemg_d_addr(c, o.pe, o.aux), (uint64_t)o.operand, o.sub);
                    }
                }
            }
            break;
        case SHMEMG_OP_WAIT_UNTIL:
            if (o.issuer == me) {
                // the leader's result decides for the whole PE (in pe_mode CLUSTER the other
                // CTAs read it through DSMEM); two slots, so the leader rewrites one only
                // after the PE barrier of the next wait, which every CTA passes after reading
                const int slot = n_waits++ & 1;
                if (threadIdx.x == 0) {
                    int w = SHMEMG_SUCCESS;
                    if (leader) w = shmemg_d_signal_wait_until(c, (const uint64_t *)shmemg_d_addr(c, me, o.dst), o.sub,
                                                               (uint64_t)o.operand, i);
                    s_wrc[slot] = w;
                }
                shmemg_d_pe_sync(c);
                rc = c.pe_mode == SHMEMG_PE_MODE_CLUSTER && c.cluster_dim > 1
                         ? shmemg_d_ld_cluster<int>(shmemg_d_cluster_addr(&s_wrc[slot], 0))
                         : s_wrc[slot];
            }
            break;
        case SHMEMG_OP_QUIET:
        case SHMEMG_OP_FENCE:  // fence on a context completes it too (ordering by completion)
            if (o.issuer == me || o.issuer < 0) {
                if (my_ctx && (o.sub == SHMEMG_CTX_ALL || o.sub == my_ctx)) ctx_drain(c, s_ctx[my_ctx - 1], ctx_ring);
                shmemg_d_quiet_pe(c);
            }
            break;
        case SHMEMG_OP_BARRIER_ALL:
            if (active) rc = shmemg_d_scope_sync(c, SHMEMG_TEAM_WORLD, i, nullptr, warp);
            break;
        case SHMEMG_OP_TEAM_SYNC: {
            int grp;
            if (active && shmemg_d_team_rank(*shmemg_d_team(c, o.team), me, &grp) >= 0)
                rc = shmemg_d_scope_sync(c, o.team, i, cs, warp);
            break;
        }
        case SHMEMG_OP_BROADCAST:
            if (staged(o)) rc = shmemg_d_cluster_broadcastmem_pe(c, s_cs, s_ring, o.dst, o.src, o.n, o.pe, i);
            else if (active) rc = shmemg_d_broadcastmem_scoped(c, o.team, o.dst, o.src, o.n, o.pe, i, cs, warp);
            break;
        case SHMEMG_OP_FCOLLECT:
            if (staged(o)) rc = shmemg_d_cluster_fcollectmem_pe(c, s_cs, s_ring, o.dst, o.src, o.n, i);
            else if (active) rc = shmemg_d_fcollectmem_scoped(c, o.team, o.dst, o.src, o.n, i, cs, warp);
            break;
        case SHMEMG_OP_ALLTOALL:
            if (staged(o)) rc = shmemg_d_cluster_alltoallmem_pe(c, s_cs, s_ring, o.dst, o.src, o.n, i);
            else if (active) rc = shmemg_d_alltoallmem_scoped(c, o.team, o.dst, o.src, o.n, i, cs, warp);
            break;
        case SHMEMG_OP_REDUCE:
            if (staged(o)) rc = shmemg_d_cluster_reduce_pe(c, s_cs, s_ring, o.dst, o.src, o.n, o.dtype, o.sub, i);
            else if (active) rc = shmemg_d_reduce_scoped(c, o.team, o.dst, o.src, o.n, o.dtype, o.sub, i, cs, warp);
            break;
        default:
            if (leader) shmemg_d_set_status(c, SHMEMG_ERR_INVALID_ARG, i);
            rc = SHMEMG_ERR_INVALID_ARG;
        }
        if (warp) {
            // the active warp's result decides for the PE (the same two-slot hand-over as a
            // wait's; in pe_mode CLUSTER the other CTAs read the leader's slot via DSMEM)
            const int slot = n_waits++ & 1;
            if (threadIdx.x == 0) s_wrc[slot] = rc;
            shmemg_d_pe_sync(c);
            rc = c.pe_mode == SHMEMG_PE_MODE_CLUSTER && c.cluster_dim > 1
                     ? shmemg_d_ld_cluster<int>(shmemg_d_cluster_addr(&s_wrc[slot], 0))
                     : s_wrc[slot];
        }
        if (rc != SHMEMG_SUCCESS) {
            failed = true;  // uniform across the PE: every thread leaves both loops
            if (!dsm) break;
        }
    }
    }
    // every context's transfers complete before the PE ends (none may still read this
    // CTA's shared memory when it exits)
    if (my_ctx) ctx_drain(c, s_ctx[my_ctx - 1], ctx_ring);
    shmemg_d_quiet_pe(c);
    if (dsm) shmemg_d_cluster_end();  // no CTA leaves while a peer may still touch its shared memory
}

int interp_threads() {
    static int t = 0;
    if (!t) {
        const char *e = getenv("SHMEMG_INTERP_THREADS");
        t = e && *e ? atoi(e) : INTERP_THREADS;
        if (t < 32 || t > INTERP_THREADS || t % 32) t = INTERP_THREADS;
    }
    return t;
}

// Cooperative launch of `kernel` with one CTA (or cluster) per PE; `threads` per CTA
// (0: the interpreter's count).
int launch_pe_grid(const void *kernel, void **args, size_t smem, cudaStream_t s, int threads) {
    State &S = st();
    if (threads <= 0) threads = interp_threads();
    const int cd = S.cluster_dim;
    const unsigned grid = S.pe_mode == SHMEMG_PE_MODE_CLUSTER ? (unsigned)(S.npes * cd) : (unsigned)S.npes;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na = 0;
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    na++;
    if (cd > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = cd;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        na++;
        int nclusters = 0;
        cudaLaunchConfig_t q = cfg;
        q.attrs = attr + 1;
        q.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &q) != cudaSuccess) {
            cudaGetLastError();
            return SHMEMG_ERR_UNSUPPORTED;
        }
        if ((int64_t)nclusters * cd < (int64_t)grid) return SHMEMG_ERR_UNSUPPORTED;
    } else {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
        if ((int64_t)per_sm * S.sm_count < (int64_t)grid) return SHMEMG_ERR_UNSUPPORTED;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    cudaError_t e = cudaLaunchKernelExC(&cfg, kernel, args);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        cudaGetLastError();
        return SHMEMG_ERR_UNSUPPORTED;
    }
    return cuda_rc(e);
}

}  // namespace shmemg

using namespace shmemg;

extern "C" int shmemg_run_script(const shmemg_op_t *ops, int64_t nops, int64_t *fetched, void *stream) {
    if (int rc = check_init()) return rc;
    if (nops < 0 || (nops && !ops)) return SHMEMG_ERR_INVALID_ARG;
    if (nops == 0) return SHMEMG_SUCCESS;
    shmemg_device_ctx_t c = device_ctx();
    // the bulk engine's shared-memory ring (disable with SHMEMG_BULK=0)
    static int bulk = -1;
    if (bulk < 0) {
        const char *e = getenv("SHMEMG_BULK");
        bulk = (e && *e == '0') ? 0 : 1;
        if (bulk && cudaFuncSetAttribute((const void *)k_interp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(SHMEMG_BULK_SMEM + CTX_SMEM)) != cudaSuccess) {
            cudaGetLastError();
            bulk = 0;
        }
    }
    int use_bulk = bulk;
    void *args[] = {(void *)&c, (void *)&ops, (void *)&nops, (void *)&fetched, (void *)&use_bulk};
    return launch_pe_grid((const void *)k_interp, args, use_bulk ? SHMEMG_BULK_SMEM + CTX_SMEM : 0, to_stream(stream));
}
