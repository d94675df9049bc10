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
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace shmemg {

constexpr int INTERP_THREADS = 512;
constexpr int OP_BATCH = 64;  // op records staged in shared memory at a time
// shared-team alltoalls staged through the DSMEM windows: at most this many bytes per
// member (P blocks).  Measured on a cluster of 8 PEs: staged 3.96 / 4.48 / 4.91 us per op
// at 64 B / 512 B / 1 KiB blocks against 5.53-5.58 us through L2, and behind from 2 KiB
// blocks (5.74 against 5.59 us)
constexpr uint64_t DSM_A2A_MAX = 8u << 10;

// ---------------------------------------------------------------- the bulk engine
// Thread 0 of every CTA moves the CTA's bulk (TMA) traffic through one ring of
// RING_STAGES shared-memory stages of RING_CHUNK bytes: a chunk is loaded global ->
// shared (cp.async.bulk, completion counted in bytes on the stage's mbarrier), then
// stored shared -> global (cp.async.bulk, bulk groups).  Two kinds of transfer share
// the ring, in ring order:
//  * queue 0, the default context's large aligned puts and gets (>= SHMEMG_BULK_MIN):
//    blocking -- the op returns once they are written.  The PE's CTAs split the chunks
//    (every ncta-th chunk) along the hardware cluster shape, so a launch without
//    clusters still copies every chunk;
//  * queues 1..3, the explicit contexts (Sec. 6.2: contexts as independent ordering and
//    completion domains, an optional resource-limited feature beside the default device
//    context): a context's put_nbi / get_nbi is queued in the PE's leader CTA and moved
//    in the background -- the engine advances at every op boundary -- and only quiet /
//    fence on that context (or on all) waits for it.  Where the GPU holds a second CTA
//    per PE, the contexts run on that CTA instead (the context agents below).
// A context alone thus keeps the whole ring in flight, like a blocking copy.  Chunk j of
// the ring uses stage j % RING_STAGES and completes phase (j / RING_STAGES) & 1 of its
// mbarrier; a stage is reloaded only after the store of its previous chunk has read it.
constexpr int RING_STAGES = 6;
constexpr uint32_t RING_CHUNK = SHMEMG_BULK_CHUNK;
constexpr size_t RING_SMEM = (size_t)RING_STAGES * RING_CHUNK;
constexpr int CTX_QCAP = 8;   // queued transfers per context
constexpr int NQ = SHMEMG_DEVICE_CTX_COUNT;  // queue 0 + one per explicit context

struct DmaXfer {
    uint64_t dst, src, n;    // generic global addresses, 16-byte multiples
    uint32_t first, stride;  // chunks first, first + stride, ... of the transfer
};
struct DmaState {
    DmaXfer q[NQ][CTX_QCAP];
    uint32_t head[NQ], tail[NQ];  // queued transfers; q[k][head] is being loaded
    uint64_t next[NQ];            // next chunk (in first + i*stride numbering, i counted) of q[k][head]
    uint64_t last[NQ];            // 1 + ring index of the queue's last chunk issued (0: none)
    uint64_t ld, st;              // ring chunks whose loads / stores are issued
    uint64_t st_dst[RING_STAGES];
    uint32_t st_len[RING_STAGES];
    uint64_t bar[RING_STAGES];
    uint32_t rr;                  // next explicit context to serve
    int dead;                     // a load never landed: nothing is issued any more
};

__device__ __forceinline__ void dma_init(DmaState &x) {
    for (int k = 0; k < NQ; k++) x.head[k] = x.tail[k] = 0, x.next[k] = x.last[k] = 0;
    x.ld = x.st = 0;
    x.rr = 0;
    x.dead = 0;
    for (int k = 0; k < RING_STAGES; k++)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shmemg_smem_u32(&x.bar[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool dma_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(shmemg_smem_u32(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

// bulk wait_group.read with a run-time count of newer groups allowed to stay pending
__device__ __forceinline__ void dma_wait_read(uint64_t newer) {
    switch (newer < RING_STAGES - 1 ? (int)newer : RING_STAGES - 1) {
    case 0: asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.bulk.wait_group.read 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.bulk.wait_group.read 4;" ::: "memory"); break;
    default: asm volatile("cp.async.bulk.wait_group.read 5;" ::: "memory"); break;
    }
}

// the next queue with a chunk to load: queue 0 first, then the contexts in turn
__device__ __forceinline__ int dma_pick(DmaState &x) {
    if (x.head[0] != x.tail[0]) return 0;
    for (int i = 0; i < NQ - 1; i++) {
        const int k = 1 + (int)((x.rr + i) % (NQ - 1));
        if (x.head[k] != x.tail[k]) {
            x.rr = (uint32_t)(k % (NQ - 1));
            return k;
        }
    }
    return -1;
}

// Issues what can be issued now without waiting: stores of chunks whose loads have
// landed, then loads into stages whose previous chunk's store has read them.
__device__ __noinline__ void dma_progress(DmaState &x, uint8_t *ring) {
    while (x.st < x.ld) {
        const uint32_t s = (uint32_t)(x.st % RING_STAGES);
        if (!dma_test(&x.bar[s], (uint32_t)((x.st / RING_STAGES) & 1))) break;
        shmemg_bulk_store((void *)x.st_dst[s], ring + (size_t)s * RING_CHUNK, x.st_len[s]);
        x.st++;
    }
    if (x.dead) return;
    while (x.ld < x.st + RING_STAGES) {
        const int k = dma_pick(x);
        if (k < 0) break;
        if (x.ld >= RING_STAGES) dma_wait_read(x.st - (x.ld - RING_STAGES) - 1);  // stores issued after that chunk's
        const DmaXfer &t = x.q[k][x.head[k] % CTX_QCAP];
        const uint64_t off = (t.first + x.next[k] * t.stride) * (uint64_t)RING_CHUNK;
        const uint32_t len = (uint32_t)(t.n - off < RING_CHUNK ? t.n - off : RING_CHUNK);
        const uint32_t s = (uint32_t)(x.ld % RING_STAGES);
        x.st_dst[s] = t.dst + off;
        x.st_len[s] = len;
        shmemg_bulk_load(ring + (size_t)s * RING_CHUNK, (const void *)(t.src + off), len, &x.bar[s]);
        x.ld++;
        x.last[k] = x.ld;
        if (off + (uint64_t)t.stride * RING_CHUNK >= t.n) {  // that was the transfer's last chunk
            x.head[k]++;
            x.next[k] = 0;
        } else {
            x.next[k]++;
        }
    }
}

// anything in flight or queued (an inline test before the out-of-line progress call)
__device__ __forceinline__ bool dma_busy(const DmaState &x) {
    bool b = x.st != x.ld;
#pragma unroll
    for (int k = 0; k < NQ; k++) b |= x.head[k] != x.tail[k];
    return b;
}

__device__ __forceinline__ bool dma_queue_done(const DmaState &x, int k) {
    return x.head[k] == x.tail[k] && x.last[k] <= x.st;
}

// Completes queue k (k < 0: every queue) -- bounded waits; a load that never lands is
// recorded as a timeout, and once the other loads in flight have landed (bounded) the
// engine stops issuing -- then makes the writes visible to generic loads.  No load is
// left writing the ring when it returns unless the status word says so (detail -4).
__device__ __noinline__ void dma_drain(const shmemg_device_ctx_t &c, DmaState &x, uint8_t *ring, int k) {
    for (;;) {
        dma_progress(x, ring);
        bool done = true;
        for (int q = 0; q < NQ; q++)
            if ((k < 0 || q == k) && !dma_queue_done(x, q)) done = false;
        if (done || (x.dead && x.st == x.ld)) break;
        if (x.st < x.ld) {
            const uint32_t s = (uint32_t)(x.st % RING_STAGES);
            if (!shmemg_mbar_wait(&x.bar[s], (uint32_t)((x.st / RING_STAGES) & 1), c.timeout_ns)) {
                const bool drained = shmemg_bulk_drain_loads(x.bar, RING_STAGES, x.st, x.ld, c.timeout_ns);
                shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, drained ? -3 : -4);
                x.dead = 1;
                if (!drained) break;
                x.st = x.ld;  // every load landed: their chunks are abandoned, the ring is free
                for (int q = 0; q < NQ; q++) x.head[q] = x.tail[q], x.next[q] = 0;
            }
        } else if (x.dead) {
            for (int q = 0; q < NQ; q++) x.head[q] = x.tail[q], x.next[q] = 0;  // nothing more is moved
        }
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");  // async-proxy writes -> generic readers
}

__device__ __noinline__ void dma_enqueue(const shmemg_device_ctx_t &c, DmaState &x, uint8_t *ring, int k,
                                            uint64_t dst, uint64_t src, uint64_t n, uint32_t first, uint32_t stride) {
    if (x.tail[k] - x.head[k] == CTX_QCAP) dma_drain(c, x, ring, k);  // queue full: finish what is queued
    if ((uint64_t)first * RING_CHUNK >= n) return;                     // no chunk of this transfer is ours
    asm volatile("fence.proxy.async.global;" ::: "memory");             // earlier generic writes -> async proxy
    x.q[k][x.tail[k] % CTX_QCAP] = {dst, src, n, first, stride};
    x.tail[k]++;
    dma_progress(x, ring);
}

// Large aligned puts and gets (>= SHMEMG_BULK_MIN) on the default context go through the
// bulk engine when the launch provides its ring (use_bulk): while no context transfer is
// queued or in flight the ring is free and the copy runs the lean blocking loop of the
// device API on it (its own mbarriers, state in registers); otherwise it joins the
// engine's queue 0 behind the chunks in flight.  The PE's other threads copy smaller or
// unaligned ones with vector loads and stores.
__device__ __forceinline__ void pe_copy(const shmemg_device_ctx_t &c, shmemg_group g, uint8_t *d, const uint8_t *s,
                                        uint64_t n, int use_bulk, uint8_t *ring, DmaState &x, uint64_t *bars) {
    if (use_bulk && n >= SHMEMG_BULK_MIN && (((uint64_t)d | (uint64_t)s | n) & 15) == 0) {
        const bool cl = c.pe_mode == SHMEMG_PE_MODE_CLUSTER;
        const uint32_t first = cl ? shmemg_d_cluster_ctarank() : 0u, stride = cl ? shmemg_d_cluster_nctarank() : 1u;
        if (threadIdx.x == 0) {
            if (!dma_busy(x)) {
                // the engine's last stores were issued; they must have read their stages
                // before the lean loop loads into them
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                shmemg_d_bulk_copy_thread_n<RING_STAGES>(c, d, s, n, first, stride, ring, bars);
            } else {
                dma_enqueue(c, x, ring, 0, (uint64_t)d, (uint64_t)s, n, first, stride);
                dma_drain(c, x, ring, 0);
            }
        }
    } else {
        shmemg_d_copy_group(g, d, s, n);
    }
}

// A context moves a transfer in the background when the bulk engine is on and the bulk
// copy's 16-byte rule holds; otherwise the op completes at once like the default
// context's (completing earlier than quiet is always allowed).
__device__ __forceinline__ bool ctx_aligned(const shmemg_device_ctx_t &, const void *d, const void *s, uint64_t n,
                                            int use_bulk) {
    return use_bulk && n > 0 && (((uint64_t)d | (uint64_t)s | n) & 15) == 0;
}

// ---------------------------------------------------------------- context agents
// A context's engine on the PE's own CTA advances only between the PE's ops and stalls the
// PE whenever the SM's copy engine is busy (its stores are read out at the SM's store
// rate, and a reload or a new bulk instruction waits for them), so it hands back in stalls
// what it gains in overlap.  When the GPU holds two CTAs per PE (CTA PEs without hardware
// clusters), each PE gets a context agent instead: a second CTA, on another SM with its
// own copy engine, whose thread 0 moves the PE's context 1..3 transfers.  The
// PE posts a context's transfer to its mailbox (the descriptor, then a release of the
// context's posted count) and goes on at once; the agent takes it (acquire), moves it
// through its own ring with the lean bulk loop, and once it is written (bulk wait_group 0,
// then the async-proxy fence) releases the context's done count.  Quiet / fence on a
// context waits (bounded) until done reaches what the PE has posted.  The PE releases
// `exit` with the launch's epoch when its script ends; the agent leaves when every
// transfer is done and exit is set.
constexpr int AGENT_MAX_PES = 128;
// Counts are tagged with the launch's epoch in their upper 32 bits, so a mailbox needs no
// reset between launches: a count left by an earlier launch reads as 0.
struct CtxMailbox {
    DmaXfer q[NQ - 1][CTX_QCAP];  // contexts 1..NQ-1; slot = count % CTX_QCAP
    uint64_t posted[NQ - 1];      // epoch:count, released by the PE
    uint64_t done[NQ - 1];        // epoch:count, released by the agent
    uint32_t exit;                // the launch's epoch, released by the PE at its end
    uint32_t beat;                // the PE's op batch, written as it walks (the agent's sign of life)
};
__device__ CtxMailbox g_mbox[AGENT_MAX_PES];
// The epoch of a launch with agents is g_agent_epoch + 1 (never 0): every CTA reads it at
// its start, and the last CTA to finish stores it back, so the next launch -- stream
// ordered after this one, a graph replay included -- uses the next epoch.
__device__ uint32_t g_agent_epoch, g_agent_exits;

__device__ __forceinline__ uint32_t mb_count(const uint64_t *p, uint32_t epoch) {
    const uint64_t v = shmemg_d_ld_acquire_u64(p);
    return (uint32_t)(v >> 32) == epoch ? (uint32_t)v : 0u;
}
__device__ __forceinline__ void mb_set(uint64_t *p, uint32_t epoch, uint32_t n) {
    shmemg_d_st_release_u64(p, ((uint64_t)epoch << 32) | n);
}

// The agent (thread 0 of the PE's agent CTA; the CTA's other threads have left) moves the
// posted transfers in order, each through the device API's lean bulk loop on the CTA's
// whole ring (the same loop as a blocking copy), and releases its context's done count
// after each one.  Waits are bounded: a load that never lands ends the lean loop with a
// timeout (status set); the ring is then left alone and later transfers are counted done
// without being moved, so no quiet waits forever.  An agent that sees no post, no new op
// batch of its PE and no exit flag for 8 x timeout_ns (longer than any bounded wait of the
// PE) records a timeout (detail -5) and leaves; a later quiet on it then times out in the PE.
__device__ __noinline__ void ctx_agent(const shmemg_device_ctx_t &c, CtxMailbox *mb, uint32_t epoch, uint8_t *ring,
                                       uint64_t *bars) {
    uint32_t taken[NQ - 1] = {}, beat = 0, nap = 128;
    bool dead = false;
    uint64_t idle_since = 0;
    for (;;) {
        bool got = false;
        for (int k = 0; k < NQ - 1; k++) {
            const uint32_t p = mb_count(&mb->posted[k], epoch);
            for (; taken[k] != p; taken[k]++) {
                const DmaXfer d = mb->q[k][taken[k] % CTX_QCAP];
                if (!dead && shmemg_d_bulk_copy_thread_n<RING_STAGES>(c, (uint8_t *)d.dst, (const uint8_t *)d.src, d.n,
                                                                       0, 1, ring, bars) != SHMEMG_SUCCESS)
                    dead = true;  // (the lean loop waited, bounded, for its loads in flight)
                mb_set(&mb->done[k], epoch, taken[k] + 1);
                got = true;
            }
        }
        if (got) {
            idle_since = 0;
            nap = 128;
            continue;
        }
        if (shmemg_d_ld_acquire_u32(&mb->exit) == epoch) {
            // the PE's posts before its exit are visible now: any the loop above did not
            // see yet are taken first
            bool late = false;
            for (int k = 0; k < NQ - 1; k++) late |= mb_count(&mb->posted[k], epoch) != taken[k];
            if (!late) break;
            continue;
        }
        const uint64_t now = shmemg_d_globaltimer();
        const uint32_t b = *(volatile uint32_t *)&mb->beat;
        if (idle_since == 0 || b != beat) idle_since = now, beat = b;
        else if (now - idle_since > 8 * c.timeout_ns) {
            shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, -5);
            break;
        }
        __nanosleep(nap);  // idle: poll less often (a post, or the end, waits at most ~1 us)
        if (nap < 1024) nap *= 2;
    }
}

// The PE's side (thread 0): post a context transfer; false if the mailbox stayed full
// for timeout_ns (status set; the transfer is not made)
__device__ __noinline__ bool agent_post(const shmemg_device_ctx_t &c, CtxMailbox *mb, uint32_t epoch, uint32_t *posted,
                                        int k, uint64_t dst, uint64_t src, uint64_t n, int64_t op_index) {
    const int q = k - 1;
    uint64_t t0 = 0;
    while (posted[q] - mb_count(&mb->done[q], epoch) >= CTX_QCAP) {
        const uint64_t now = shmemg_d_globaltimer();
        if (t0 == 0) t0 = now;
        else if (now - t0 > c.timeout_ns) {
            shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, op_index);
            return false;
        }
        __nanosleep(128);
    }
    mb->q[q][posted[q] % CTX_QCAP] = {dst, src, n, 0, 1};
    __threadfence();  // the descriptor, and the PE's writes before this op, before the count
    mb_set(&mb->posted[q], epoch, ++posted[q]);
    return true;
}

// The PE's side (thread 0): wait until context k (k = SHMEMG_CTX_ALL: every context) has
// written everything posted to it; bounded by timeout_ns (status set)
__device__ __noinline__ void agent_quiet(const shmemg_device_ctx_t &c, CtxMailbox *mb, uint32_t epoch,
                                         const uint32_t *posted, int k, int64_t op_index) {
    uint64_t t0 = 0;
    for (int q = 0; q < NQ - 1; q++) {
        if (k != SHMEMG_CTX_ALL && q != k - 1) continue;
        while (mb_count(&mb->done[q], epoch) != posted[q]) {
            const uint64_t now = shmemg_d_globaltimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > c.timeout_ns) {
                shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, op_index);
                return;
            }
            __nanosleep(64);
        }
    }
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

// with_agents: the launch has 2 x npes CTAs, CTA npes + p being PE p's context agent
__global__ void __launch_bounds__(INTERP_THREADS) k_interp(shmemg_device_ctx_t c, const shmemg_op_t *ops,
                                                           int64_t nops, int64_t *fetched, int use_bulk,
                                                           int with_agents) {
    const int me = shmemg_d_my_pe(c);
    const shmemg_group g = shmemg_d_group_pe(c);
    const bool leader = shmemg_d_pe_leader(c);
    __shared__ int s_wrc[2];
    int n_waits = 0;
    extern __shared__ __align__(128) uint8_t s_ring[];
    __shared__ __align__(8) uint64_t s_bars[RING_STAGES];  // the lean blocking loop's mbarriers
    // the op list is staged through shared memory OP_BATCH records at a time (one
    // coalesced copy per batch instead of a dependent global load per op and thread)
    __shared__ __align__(16) shmemg_op_t s_ops[OP_BATCH];
    // per op of the batch, decoded once by warp 0: 0 = nothing for this PE, 1 = run, 2 = invalid;
    // and the indices of the ops with a nonzero code, in order
    __shared__ uint8_t s_act[OP_BATCH];
    __shared__ uint8_t s_list[OP_BATCH];
    __shared__ int s_nact;
    // shared-team ops of a CTA-mode heap launched in clusters run inside the cluster: the
    // team barrier is the hardware cluster barrier, small alltoalls are staged in the
    // bulk ring, which then serves as each CTA's DSMEM window (free between ops: every
    // bulk copy has drained)
    __shared__ shmemg_cluster_state_t s_cs;
    // the bulk engine (thread 0 only; with the launch's ring): the default context's
    // large copies and, in the PE's leader CTA, the explicit contexts' queues
    __shared__ __align__(16) DmaState s_dma;
    uint32_t agent_epoch = 0;
    if (with_agents) {
        agent_epoch = *(volatile uint32_t *)&g_agent_epoch + 1u;
        if (agent_epoch == 0) agent_epoch = 1;
    }
    // (thread 0 of each CTA, at its end: the last one moves the epoch on)
    auto agent_exit = [&]() {
        __threadfence();
        if (atomicAdd(&g_agent_exits, 1u) == gridDim.x - 1) {
            g_agent_exits = 0;
            g_agent_epoch = agent_epoch;
            __threadfence();
        }
    };
    if (with_agents && blockIdx.x >= (uint32_t)c.npes) {  // a context agent, not a PE
        if (threadIdx.x == 0) {
            ctx_agent(c, &g_mbox[blockIdx.x - (uint32_t)c.npes], agent_epoch, s_ring, s_bars);
            agent_exit();
        }
        return;
    }
    CtxMailbox *const mb = with_agents ? &g_mbox[me] : nullptr;  // this PE's contexts go to its agent
    uint32_t ag_posted[NQ - 1] = {};                              // (thread 0's counts)
    const bool dma = use_bulk && threadIdx.x == 0;
    const bool ctx_home = use_bulk && shmemg_d_pe_leader_cta(c);  // this CTA serves the PE's contexts
    if (dma) dma_init(s_dma);
    // (only when the launch really has clusters of cluster_dim CTAs: a launch without
    // them -- a profiler replaying it, say -- runs the shared team on the L2/HBM path and
    // never maps a peer CTA that does not exist)
    const bool dsm = c.pe_mode == SHMEMG_PE_MODE_CTA && c.cluster_dim > 1 &&
                     shmemg_d_cluster_nctarank() == (uint32_t)c.cluster_dim;
    shmemg_cluster_state_t *cs = dsm ? &s_cs : nullptr;
    const uint64_t win_bytes = use_bulk ? SHMEMG_BULK_SMEM : 0;
    if (dsm) shmemg_d_cluster_begin(s_cs);
    // Which shared-team collectives are staged through the DSMEM windows: alltoalls of at
    // most DSM_A2A_MAX bytes per member.  Every other shared-team collective moves its data
    // through L2 between cluster barriers -- measured faster at every size, because a staged
    // op copies its source twice (into the window, then out of the peers' windows over the
    // SM-to-SM network, whose per-SM port a broadcast's root serialises) and needs a third
    // cluster barrier, while the hardware barrier is what makes the shared team fast.
    auto staged = [&](const shmemg_op_t &o) {
        if (!dsm || o.team != SHMEMG_TEAM_SHARED || o.kind != SHMEMG_OP_ALLTOALL) return false;
        const uint64_t b = o.n * (uint64_t)c.cluster_dim;
        return b > 0 && b <= DSM_A2A_MAX && b <= win_bytes;
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
    if (mb && threadIdx.x == 0) *(volatile uint32_t *)&mb->beat = (uint32_t)(base / OP_BATCH) + 1;
    __syncthreads();
    for (int q = threadIdx.x; q < cnt * 4; q += blockDim.x)
        reinterpret_cast<uint4 *>(s_ops)[q] = __ldcg(reinterpret_cast<const uint4 *>(ops + base) + q);
    __syncthreads();
    // validity and participation once per op and CTA, not once per op and thread, and the
    // batch's ops this PE takes part in as a compact list (in order): the PE walks only
    // those, and the ops of other PEs cost it nothing
    if (threadIdx.x < 32) {
        const int lane = (int)threadIdx.x;
        int nact = 0;
        for (int k0 = 0; k0 < cnt; k0 += 32) {
            const int k = k0 + lane;
            int a = 0;
            if (k < cnt) {
                a = !op_valid(c, s_ops[k]) ? 2 : op_involves(s_ops[k], me) ? 1 : 0;
                s_act[k] = (uint8_t)a;
            }
            const unsigned m = __ballot_sync(0xffffffffu, a != 0);
            if (a != 0) s_list[nact + __popc(m & ((1u << lane) - 1u))] = (uint8_t)k;
            nact += __popc(m);
        }
        if (lane == 0) s_nact = nact;
    }
    __syncthreads();
    if (dma && dma_busy(s_dma)) dma_progress(s_dma, s_ring);  // background transfers advance
    const int nact = s_nact;
    // the PE's ops in order; once failed (only in a clustered CTA-mode launch) every
    // remaining op of the script, for its cluster barriers
    for (int qi = 0, k_next = 0;;) {
        int k;
        if (!failed) {
            if (qi >= nact) break;
            k = s_list[qi++];
        } else {
            if (!dsm || k_next >= cnt) break;
            k = k_next;
        }
        k_next = k + 1;
        const int64_t i = base + k;
        if (dma && dma_busy(s_dma)) dma_progress(s_dma, s_ring);  // background transfers advance
        const int act = s_act[k];
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
        if (staged(o)) {
            // the ring becomes this CTA's DSMEM window: no background chunk may still be in
            // it (every CTA of the cluster drains before the collective's entry barrier, so
            // no peer writes into a window still in use)
            if (dma) dma_drain(c, s_dma, s_ring, -1);
            __syncthreads();
        }
        switch (o.kind & SHMEMG_OP_KIND_MASK) {
        case SHMEMG_OP_PUT:
        case SHMEMG_OP_PUT_NBI:
            if (o.issuer == me && o.kind == SHMEMG_OP_PUT_NBI && o.sub != 0 &&
                ctx_aligned(c, shmemg_d_addr(c, o.pe, o.dst), shmemg_d_addr(c, me, o.src), o.n, use_bulk)) {
                if (mb) {  // posted to the PE's agent
                    if (threadIdx.x == 0)
                        agent_post(c, mb, agent_epoch, ag_posted, o.sub, (uint64_t)shmemg_d_addr(c, o.pe, o.dst),
                                   (uint64_t)shmemg_d_addr(c, me, o.src), o.n, i);
                } else if (dma && ctx_home) {  // queued on its context, moved in the background
                    dma_enqueue(c, s_dma, s_ring, o.sub, (uint64_t)shmemg_d_addr(c, o.pe, o.dst),
                                (uint64_t)shmemg_d_addr(c, me, o.src), o.n, 0, 1);
                }
            } else if (o.issuer == me) {
                if (warp) {
                    if (active) shmemg_d_copy_group(gw, shmemg_d_addr(c, o.pe, o.dst), shmemg_d_addr(c, me, o.src), o.n);
                } else {
                    pe_copy(c, g, shmemg_d_addr(c, o.pe, o.dst), shmemg_d_addr(c, me, o.src), o.n, use_bulk, s_ring,
                            s_dma, s_bars);
                    if (o.kind == SHMEMG_OP_PUT) shmemg_d_pe_sync(c);
                }
            }
            break;
        case SHMEMG_OP_GET:
        case SHMEMG_OP_GET_NBI:
            if (o.issuer == me && o.kind == SHMEMG_OP_GET_NBI && o.sub != 0 &&
                ctx_aligned(c, shmemg_d_addr(c, me, o.dst), shmemg_d_addr(c, o.pe, o.src), o.n, use_bulk)) {
                if (mb) {
                    if (threadIdx.x == 0)
                        agent_post(c, mb, agent_epoch, ag_posted, o.sub, (uint64_t)shmemg_d_addr(c, me, o.dst),
                                   (uint64_t)shmemg_d_addr(c, o.pe, o.src), o.n, i);
                } else if (dma && ctx_home) {
                    dma_enqueue(c, s_dma, s_ring, o.sub, (uint64_t)shmemg_d_addr(c, me, o.dst),
                                (uint64_t)shmemg_d_addr(c, o.pe, o.src), o.n, 0, 1);
                }
            } else if (o.issuer == me) {
                if (warp) {
                    if (active) shmemg_d_copy_group(gw, shmemg_d_addr(c, me, o.dst), shmemg_d_addr(c, o.pe, o.src), o.n);
                } else {
                    pe_copy(c, g, shmemg_d_addr(c, me, o.dst), shmemg_d_addr(c, o.pe, o.src), o.n, use_bulk, s_ring,
                            s_dma, s_bars);
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
                if (mb) {
                    if (threadIdx.x == 0 && o.sub != 0) agent_quiet(c, mb, agent_epoch, ag_posted, o.sub, i);
                } else if (dma && ctx_home && o.sub != 0) {
                    dma_drain(c, s_dma, s_ring, o.sub == SHMEMG_CTX_ALL ? -1 : o.sub);
                }
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
            if (active) rc = shmemg_d_broadcastmem_scoped(c, o.team, o.dst, o.src, o.n, o.pe, i, cs, warp);
            break;
        case SHMEMG_OP_FCOLLECT:
            if (active) rc = shmemg_d_fcollectmem_scoped(c, o.team, o.dst, o.src, o.n, i, cs, warp);
            break;
        case SHMEMG_OP_ALLTOALL:
            if (staged(o)) rc = shmemg_d_cluster_alltoallmem_pe(c, s_cs, s_ring, o.dst, o.src, o.n, i);
            else if (active) rc = shmemg_d_alltoallmem_scoped(c, o.team, o.dst, o.src, o.n, i, cs, warp);
            break;
        case SHMEMG_OP_REDUCE:
            if (active) rc = shmemg_d_reduce_scoped(c, o.team, o.dst, o.src, o.n, o.dtype, o.sub, i, cs, warp);
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
    // CTA's shared memory when it exits); the agent finishes its own before it leaves
    if (dma) dma_drain(c, s_dma, s_ring, -1);
    if (mb && threadIdx.x == 0) shmemg_d_st_release_u32(&mb->exit, agent_epoch);
    shmemg_d_quiet_pe(c);
    if (dsm) shmemg_d_cluster_end();  // no CTA leaves while a peer may still touch its shared memory
    if (with_agents && threadIdx.x == 0) agent_exit();
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

// Cooperative launch of `kernel` with one CTA (or cluster) per PE, grid_mult times over;
// `threads` per CTA (0: the interpreter's count).
int launch_pe_grid(const void *kernel, void **args, size_t smem, cudaStream_t s, int threads, int grid_mult) {
    State &S = st();
    if (threads <= 0) threads = interp_threads();
    const int cd = S.cluster_dim;
    const unsigned grid =
        (S.pe_mode == SHMEMG_PE_MODE_CLUSTER ? (unsigned)(S.npes * cd) : (unsigned)S.npes) * (unsigned)grid_mult;
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
    }
    // whether the GPU holds the whole grid at once: an occupancy query per kernel shape,
    // cached (a query per launch cost more host time than a small script runs)
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t, int, unsigned, int>, bool> fits;
    const auto key = std::make_tuple(kernel, threads, smem, cd, grid, S.device);
    bool ok;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = fits.find(key);
        if (it != fits.end()) {
            ok = it->second;
        } else {
            if (cd > 1) {
                int nclusters = 0;
                cudaLaunchConfig_t q = cfg;
                q.attrs = attr + 1;
                q.numAttrs = 1;
                if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &q) != cudaSuccess) {
                    cudaGetLastError();
                    nclusters = 0;
                }
                ok = (int64_t)nclusters * cd >= (int64_t)grid;
            } else {
                int per_sm = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
                ok = (int64_t)per_sm * S.sm_count >= (int64_t)grid;
            }
            fits[key] = ok;
        }
    }
    if (!ok) return SHMEMG_ERR_UNSUPPORTED;
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
                                         (int)RING_SMEM) != cudaSuccess) {
            cudaGetLastError();
            bulk = 0;
        }
    }
    int use_bulk = bulk;
    // context agents: CTA PEs without hardware clusters, when the GPU holds two CTAs per PE
    // (SHMEMG_CTX_AGENTS=0 keeps the contexts on the PE's own engine)
    static int agents = -1;
    if (agents < 0) {
        const char *e = getenv("SHMEMG_CTX_AGENTS");
        agents = (e && *e == '0') ? 0 : 1;
    }
    State &S = st();
    int with_agents = 0;
    if (agents && use_bulk && S.pe_mode == SHMEMG_PE_MODE_CTA && S.cluster_dim == 1 && S.npes <= AGENT_MAX_PES &&
        ctas_for((const void *)k_interp, interp_threads(), RING_SMEM) >= 2 * S.npes)
        with_agents = 1;
    void *args[] = {(void *)&c, (void *)&ops, (void *)&nops, (void *)&fetched, (void *)&use_bulk, (void *)&with_agents};
    return launch_pe_grid((const void *)k_interp, args, use_bulk ? RING_SMEM : 0, to_stream(stream), 0,
                          with_agents ? 2 : 1);
}
