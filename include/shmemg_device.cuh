/*
 * shmemg_device.cuh -- device API of the one-GPU symmetric heap (sm_103a).
 *
 * Device-initiated operations (paper Sec. 6.3, "device-initiated path"): device code
 * addresses PE p's copy of a symmetric object as heap + p*H + offset, without per-op
 * pointer classification (Sec. 6.3: "should not require device code to perform
 * dynamic pointer classification").  Scopes (Sec. 6.3, participation scopes):
 *   thread  -- one thread issues the operation;
 *   group   -- every thread of a shmemg_group (warp, block, cluster or grid) calls with
 *              identical arguments (uniform participation, Sec. 6.3 normative excerpt)
 *              and the work is split among them.
 * Ordering (Sec. 6.4): fence orders, quiet completes the caller's operations; data
 * moved with plain stores is complete once a GPU-scope fence follows it; bulk (TMA)
 * stores also need their bulk group drained and a proxy fence.  Every wait is bounded
 * by ctx.timeout_ns of %globaltimer; on expiry the first error is recorded in the
 * device status word and the wait returns SHMEMG_ERR_TIMEOUT (no trap, no hang).
 */
#ifndef SHMEMG_DEVICE_CUH
#define SHMEMG_DEVICE_CUH

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "shmemg.h"

/* ------------------------------------------------------------ reserved prefix layout */
#define SHMEMG_STATUS_OFF 0ull            /* int32 code, int32 pad, int64 detail */
#define SHMEMG_TEAMS_OFF 4096ull          /* SHMEMG_MAX_TEAMS x shmemg_dteam_t */
#define SHMEMG_BARRIERS_OFF (256ull << 10) /* SHMEMG_MAX_BARRIERS x shmemg_dbar_t */
#define SHMEMG_MAX_BARRIERS 65536u
#define SHMEMG_SCRATCH_OFF (2ull << 20)   /* library scratch words (2 MiB) */

typedef struct {
    int32_t start, stride, size;  /* members start + r*stride (+ group*gstride) */
    int32_t ngroups, gstride;     /* SHARED: one group per cluster */
    int32_t bar_base;             /* barrier slot of group 0 */
    int32_t valid, pad;
} shmemg_dteam_t;

typedef struct {
    uint32_t count;
    uint32_t gen;
    uint32_t pad[30];             /* one 128-byte line per barrier */
} shmemg_dbar_t;

typedef struct {
    uint32_t rank;   /* this thread's rank in the cooperating group */
    uint32_t size;   /* threads in the group */
} shmemg_group;

/* ------------------------------------------------------------------ PTX helpers */
static __device__ __forceinline__ uint64_t shmemg_d_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
static __device__ __forceinline__ void shmemg_d_fence_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
static __device__ __forceinline__ void shmemg_d_fence_sys() {
    asm volatile("fence.acq_rel.sys;" ::: "memory");
}
static __device__ __forceinline__ uint64_t shmemg_d_ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ uint32_t shmemg_d_ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ uint64_t shmemg_d_ld_acquire_sys_u64(const volatile uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ void shmemg_d_st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
static __device__ __forceinline__ void shmemg_d_st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
static __device__ __forceinline__ void shmemg_d_red_release_add_u64(uint64_t *p, uint64_t v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
static __device__ __forceinline__ uint32_t shmemg_d_cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
static __device__ __forceinline__ uint32_t shmemg_d_cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
/* All threads of all CTAs of the cluster; release/acquire at cluster scope. */
static __device__ __forceinline__ void shmemg_d_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

/* ------------------------------------------------------------------ context access */
static __device__ __forceinline__ uint8_t *shmemg_d_addr(const shmemg_device_ctx_t &c, int pe, uint64_t off) {
    return c.heap + (uint64_t)pe * c.pe_stride + off;
}
static __device__ __forceinline__ uint64_t shmemg_d_offset(const shmemg_device_ctx_t &c, const void *sym) {
    return (uint64_t)((const uint8_t *)sym - c.heap);
}
/* shmem_ptr analogue: device address of `sym` on `pe` (valid in device code only). */
static __device__ __forceinline__ void *shmemg_d_ptr(const shmemg_device_ctx_t &c, const void *sym, int pe) {
    return shmemg_d_addr(c, pe, shmemg_d_offset(c, sym));
}
static __device__ __forceinline__ int shmemg_d_n_pes(const shmemg_device_ctx_t &c) { return c.npes; }
/* PE of the calling thread: its CTA (pe_mode CTA) or its cluster (pe_mode CLUSTER),
 * for a 1-D grid launched with the library's PE layout. */
static __device__ __forceinline__ int shmemg_d_my_pe(const shmemg_device_ctx_t &c) {
    return c.pe_mode == SHMEMG_PE_MODE_CLUSTER ? (int)(blockIdx.x / (uint32_t)c.cluster_dim) : (int)blockIdx.x;
}
static __device__ __forceinline__ const shmemg_dteam_t *shmemg_d_team(const shmemg_device_ctx_t &c, int team) {
    return (const shmemg_dteam_t *)(c.state + SHMEMG_TEAMS_OFF) + team;
}
/* Team rank of world PE `pe` in `team` and its group index; -1 if not a member. */
static __device__ __forceinline__ int shmemg_d_team_rank(const shmemg_dteam_t &t, int pe, int *group) {
    int rel = pe - t.start;
    if (rel < 0) return -1;
    int g = t.gstride > 0 ? rel / t.gstride : 0;
    if (g >= t.ngroups) return -1;
    rel -= g * t.gstride;
    if (rel % t.stride) return -1;
    int r = rel / t.stride;
    if (r >= t.size) return -1;
    if (group) *group = g;
    return r;
}
static __device__ __forceinline__ int shmemg_d_team_member(const shmemg_dteam_t &t, int group, int r) {
    return t.start + group * t.gstride + r * t.stride;
}

/* ------------------------------------------------------------------ groups */
static __device__ __forceinline__ shmemg_group shmemg_d_group_thread() { return {0u, 1u}; }
static __device__ __forceinline__ shmemg_group shmemg_d_group_warp() { return {threadIdx.x & 31u, 32u}; }
static __device__ __forceinline__ shmemg_group shmemg_d_group_block() { return {threadIdx.x, blockDim.x}; }
static __device__ __forceinline__ shmemg_group shmemg_d_group_cluster() {
    return {shmemg_d_cluster_ctarank() * blockDim.x + threadIdx.x, shmemg_d_cluster_nctarank() * blockDim.x};
}
static __device__ __forceinline__ shmemg_group shmemg_d_group_grid() {
    return {blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x};
}
/* the whole calling PE: its block, or its cluster in pe_mode CLUSTER */
static __device__ __forceinline__ shmemg_group shmemg_d_group_pe(const shmemg_device_ctx_t &c) {
    return c.pe_mode == SHMEMG_PE_MODE_CLUSTER ? shmemg_d_group_cluster() : shmemg_d_group_block();
}
static __device__ __forceinline__ void shmemg_d_pe_sync(const shmemg_device_ctx_t &c) {
    if (c.pe_mode == SHMEMG_PE_MODE_CLUSTER) shmemg_d_cluster_sync();
    else __syncthreads();
}
/* the PE's first CTA (its only CTA in pe_mode CTA) */
static __device__ __forceinline__ bool shmemg_d_pe_leader_cta(const shmemg_device_ctx_t &c) {
    return c.pe_mode != SHMEMG_PE_MODE_CLUSTER || shmemg_d_cluster_ctarank() == 0;
}
static __device__ __forceinline__ bool shmemg_d_pe_leader(const shmemg_device_ctx_t &c) {
    return threadIdx.x == 0 && (c.pe_mode != SHMEMG_PE_MODE_CLUSTER || shmemg_d_cluster_ctarank() == 0);
}

/* ------------------------------------------------------------------ status word */
/* Records the first device-side error (later ones are dropped). */
static __device__ __forceinline__ void shmemg_d_set_status(const shmemg_device_ctx_t &c, int code, int64_t detail) {
    int *st = (int *)(c.state + SHMEMG_STATUS_OFF);
    if (atomicCAS(st, 0, code) == 0) {
        *(volatile int64_t *)(c.state + SHMEMG_STATUS_OFF + 8) = detail;
        shmemg_d_fence_gpu();
    }
}
static __device__ __forceinline__ int shmemg_d_get_status(const shmemg_device_ctx_t &c) {
    return *(volatile int *)(c.state + SHMEMG_STATUS_OFF);
}

/* ------------------------------------------------------------------ data movement */
template <typename V>
static __device__ __forceinline__ V shmemg_ld_cg(const V *p);
template <> __device__ __forceinline__ uint4 shmemg_ld_cg<uint4>(const uint4 *p) { return __ldcg(p); }
template <> __device__ __forceinline__ uint2 shmemg_ld_cg<uint2>(const uint2 *p) { return __ldcg(p); }
template <> __device__ __forceinline__ uint32_t shmemg_ld_cg<uint32_t>(const uint32_t *p) { return __ldcg(p); }
template <> __device__ __forceinline__ uint16_t shmemg_ld_cg<uint16_t>(const uint16_t *p) {
    return __ldcg((const unsigned short *)p);
}
template <> __device__ __forceinline__ uint8_t shmemg_ld_cg<uint8_t>(const uint8_t *p) {
    return (uint8_t)__ldcg((const unsigned char *)p);
}
template <> __device__ __forceinline__ int4 shmemg_ld_cg<int4>(const int4 *p) { return __ldcg(p); }
template <> __device__ __forceinline__ longlong2 shmemg_ld_cg<longlong2>(const longlong2 *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float4 shmemg_ld_cg<float4>(const float4 *p) { return __ldcg(p); }
template <> __device__ __forceinline__ int32_t shmemg_ld_cg<int32_t>(const int32_t *p) { return __ldcg(p); }
template <> __device__ __forceinline__ int64_t shmemg_ld_cg<int64_t>(const int64_t *p) {
    return (int64_t)__ldcg((const long long *)p);
}
template <> __device__ __forceinline__ float shmemg_ld_cg<float>(const float *p) { return __ldcg(p); }

/* Group-wide copy of nvec vectors of type V; each thread keeps 4 loads in flight. */
template <typename V>
static __device__ __forceinline__ void shmemg_d_copy_vec(shmemg_group g, V *dst, const V *src, uint64_t nvec) {
    uint64_t i = g.rank;
    const uint64_t s = g.size;
    for (; i + 3 * s < nvec; i += 4 * s) {
        V a = shmemg_ld_cg(src + i), b = shmemg_ld_cg(src + i + s);
        V d = shmemg_ld_cg(src + i + 2 * s), e = shmemg_ld_cg(src + i + 3 * s);
        dst[i] = a;
        dst[i + s] = b;
        dst[i + 2 * s] = d;
        dst[i + 3 * s] = e;
    }
    for (; i < nvec; i += s) dst[i] = shmemg_ld_cg(src + i);
}

/* widest power-of-two vector (<= 16 bytes) that both addresses and the length allow */
static __device__ __forceinline__ int shmemg_d_vec_width(const void *a, const void *b, uint64_t n) {
    uint64_t m = (uint64_t)a | (uint64_t)b | n;
    return (m & 15) == 0 ? 16 : (m & 7) == 0 ? 8 : (m & 3) == 0 ? 4 : (m & 1) == 0 ? 2 : 1;
}

/* Group-wide byte copy dst <- src (no overlap).  src must be global memory (the loads
 * are ld.global.cg); dst may be global or the caller's own shared memory. */
static __device__ __forceinline__ void shmemg_d_copy_group(shmemg_group g, void *dst, const void *src, uint64_t n) {
    switch (shmemg_d_vec_width(dst, src, n)) {
    case 16: shmemg_d_copy_vec(g, (uint4 *)dst, (const uint4 *)src, n / 16); break;
    case 8: shmemg_d_copy_vec(g, (uint2 *)dst, (const uint2 *)src, n / 8); break;
    case 4: shmemg_d_copy_vec(g, (uint32_t *)dst, (const uint32_t *)src, n / 4); break;
    case 2: shmemg_d_copy_vec(g, (uint16_t *)dst, (const uint16_t *)src, n / 2); break;
    default: shmemg_d_copy_vec(g, (uint8_t *)dst, (const uint8_t *)src, n); break;
    }
}

/* ------------------------------------------------------------------ bulk (TMA) copies */
/* Large aligned copies go through the Tensor Memory Accelerator's non-tensor bulk path:
 * one thread streams chunks global -> shared (cp.async.bulk, completion counted in bytes
 * on an mbarrier) and shared -> global (cp.async.bulk, bulk groups) through a ring of
 * SHMEMG_BULK_STAGES shared-memory stages, so each SM keeps several chunks in flight
 * without occupying registers.  Generic-proxy writes made before the copy are made
 * visible to the async proxy first, and the copy's writes to the generic proxy after. */
#define SHMEMG_BULK_STAGES 4
#define SHMEMG_BULK_CHUNK (32u << 10)
#define SHMEMG_BULK_SMEM (SHMEMG_BULK_STAGES * SHMEMG_BULK_CHUNK)
#define SHMEMG_BULK_MIN (64u << 10) /* smaller copies use vector loads and stores */

static __device__ __forceinline__ uint32_t shmemg_smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
static __device__ __forceinline__ void shmemg_bulk_load(void *smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(shmemg_smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     shmemg_smem_u32(smem)),
                 "l"(src), "r"(bytes), "r"(shmemg_smem_u32(bar))
                 : "memory");
}
static __device__ __forceinline__ void shmemg_bulk_store(void *dst, const void *smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(shmemg_smem_u32(smem)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
/* bounded wait for an mbarrier phase: false after ~timeout_ns */
static __device__ __forceinline__ bool shmemg_mbar_wait(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(shmemg_smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 255) == 255) {
            const uint64_t now = shmemg_d_globaltimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > timeout_ns) return false;
        }
    }
}

/* The ring invariant on the timeout path.  A ring of `stages` stages whose wait for chunk
 * j timed out still has the loads of chunks j .. min(j + stages, count) - 1 issued and not
 * waited for; they write into shared memory asynchronously, and the bulk-group wait does
 * not cover them (mbarriers track them).  This waits for each (bounded), so that after a
 * true return no load of the ring is in flight and the ring may be reused or the CTA may
 * exit.  A false return means a load did not land within another timeout: the caller
 * records it (status detail -4: the launch's results are void) and issues nothing more
 * into that ring. */
static __device__ __forceinline__ bool shmemg_bulk_drain_loads(uint64_t *bars, uint32_t stages, uint64_t j,
                                                               uint64_t count, uint64_t timeout_ns) {
    bool ok = true;
    const uint64_t end = j + stages < count ? j + stages : count;
    for (uint64_t k = j; k < end; k++)
        ok = shmemg_mbar_wait(&bars[k % stages], (uint32_t)((k / stages) & 1u), timeout_ns) && ok;
    return ok;
}

/* Thread-scope bulk copy of the chunks first, first+stride, ... of (dst <- src, n bytes);
 * dst, src and n multiples of 16.  smem: STAGES x SHMEMG_BULK_CHUNK bytes (128-byte
 * aligned); bars: STAGES mbarriers.  Returns once the data is written (blocking put
 * semantics); SHMEMG_ERR_TIMEOUT (recorded in the status word) if a stage never fills, after
 * waiting (bounded) for the loads still in flight (shmemg_bulk_drain_loads).
 * A stage is refilled one chunk behind: after chunk j's store is issued, the stage of
 * chunk j - 1 takes chunk j - 1 + STAGES once that older store has read it (bulk
 * wait_group.read 1), so the wait rarely blocks and STAGES - 1 loads stay in flight. */
template <int STAGES>
static __device__ int shmemg_d_bulk_copy_thread_n(const shmemg_device_ctx_t &c, uint8_t *dst, const uint8_t *src,
                                                  uint64_t n, uint32_t first, uint32_t stride, uint8_t *smem,
                                                  uint64_t *bars) {
    static_assert(STAGES >= 2, "a chunk is refilled one stage behind");
    const uint64_t nch = (n + SHMEMG_BULK_CHUNK - 1) / SHMEMG_BULK_CHUNK;
    if (first >= nch) return SHMEMG_SUCCESS;
    const uint32_t count = (uint32_t)((nch - first + stride - 1) / stride);
    for (int s = 0; s < STAGES; s++)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shmemg_smem_u32(&bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");  /* earlier generic writes -> async proxy */
    auto chunk = [&](uint32_t j, uint64_t *off) -> uint32_t {
        *off = (uint64_t)(first + (uint64_t)j * stride) * SHMEMG_BULK_CHUNK;
        const uint64_t left = n - *off;
        return (uint32_t)(left < SHMEMG_BULK_CHUNK ? left : SHMEMG_BULK_CHUNK);
    };
    for (uint32_t j = 0; j < count && j < STAGES; j++) {
        uint64_t off;
        const uint32_t b = chunk(j, &off);
        shmemg_bulk_load(smem + (uint64_t)j * SHMEMG_BULK_CHUNK, src + off, b, &bars[j]);
    }
    int rc = SHMEMG_SUCCESS;
    for (uint32_t j = 0; j < count; j++) {
        const uint32_t s = j % STAGES;
        if (!shmemg_mbar_wait(&bars[s], (j / STAGES) & 1u, c.timeout_ns)) {
            /* loads issued so far: chunks 0 .. j + STAGES - 2 (the refill of iteration j - 1
             * took chunk j - 2 + STAGES); those from j on are still in flight */
            const uint32_t issued = j + STAGES - 1 < count ? j + STAGES - 1 : count;
            const bool drained = shmemg_bulk_drain_loads(bars, STAGES, j, issued, c.timeout_ns);
            shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, drained ? -2 : -4);
            rc = SHMEMG_ERR_TIMEOUT;
            break;
        }
        uint64_t off;
        const uint32_t b = chunk(j, &off);
        shmemg_bulk_store(dst + off, smem + (uint64_t)s * SHMEMG_BULK_CHUNK, b);
        if (j >= 1 && j - 1 + STAGES < count) {
            /* the stage of chunk j - 1, once its store (the group before this one) has read it */
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            const uint32_t sp = (j - 1) % STAGES;
            uint64_t off2;
            const uint32_t b2 = chunk(j - 1 + STAGES, &off2);
            shmemg_bulk_load(smem + (uint64_t)sp * SHMEMG_BULK_CHUNK, src + off2, b2, &bars[sp]);
        }
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");  /* async-proxy writes -> generic readers */
    return rc;
}
static __device__ int shmemg_d_bulk_copy_thread(const shmemg_device_ctx_t &c, uint8_t *dst, const uint8_t *src,
                                                uint64_t n, uint32_t first, uint32_t stride, uint8_t *smem,
                                                uint64_t *bars) {
    return shmemg_d_bulk_copy_thread_n<SHMEMG_BULK_STAGES>(c, dst, src, n, first, stride, smem, bars);
}

/* ------------------------------------------------------------------ RMA (Sec. 2.1) */
/* put: n bytes of the caller PE's `src` -> `dst` on `pe`.  Group scope: every thread
 * of g calls with the same arguments.  On return the caller's threads have read the
 * source (local completion); remote visibility needs quiet (Sec. 6.3). */
static __device__ __forceinline__ void shmemg_d_putmem_group(const shmemg_device_ctx_t &c, shmemg_group g,
                                                             void *dst, const void *src, uint64_t n, int pe,
                                                             int my_pe) {
    shmemg_d_copy_group(g, shmemg_d_ptr(c, dst, pe), shmemg_d_ptr(c, src, my_pe), n);
}
/* get: n bytes of `src` on `pe` -> the caller PE's `dst`. */
static __device__ __forceinline__ void shmemg_d_getmem_group(const shmemg_device_ctx_t &c, shmemg_group g,
                                                             void *dst, const void *src, uint64_t n, int pe,
                                                             int my_pe) {
    shmemg_d_copy_group(g, shmemg_d_ptr(c, dst, my_pe), shmemg_d_ptr(c, src, pe), n);
}
/* block-scope forms for pe_mode CTA (the calling block is the PE) */
static __device__ __forceinline__ void shmemg_d_putmem_block(const shmemg_device_ctx_t &c, void *dst,
                                                             const void *src, uint64_t n, int pe) {
    shmemg_d_putmem_group(c, shmemg_d_group_block(), dst, src, n, pe, shmemg_d_my_pe(c));
    __syncthreads();
}
static __device__ __forceinline__ void shmemg_d_getmem_block(const shmemg_device_ctx_t &c, void *dst,
                                                             const void *src, uint64_t n, int pe) {
    shmemg_d_getmem_group(c, shmemg_d_group_block(), dst, src, n, pe, shmemg_d_my_pe(c));
    __syncthreads();
}
/* warp-scope forms: the 32 lanes of the calling warp share the copy; the warp's local
 * completion (its lanes have read the source) on return */
static __device__ __forceinline__ void shmemg_d_putmem_warp(const shmemg_device_ctx_t &c, void *dst,
                                                            const void *src, uint64_t n, int pe) {
    shmemg_d_putmem_group(c, shmemg_d_group_warp(), dst, src, n, pe, shmemg_d_my_pe(c));
    __syncwarp();
}
static __device__ __forceinline__ void shmemg_d_getmem_warp(const shmemg_device_ctx_t &c, void *dst,
                                                            const void *src, uint64_t n, int pe) {
    shmemg_d_getmem_group(c, shmemg_d_group_warp(), dst, src, n, pe, shmemg_d_my_pe(c));
    __syncwarp();
}
/* thread-scope forms */
static __device__ __forceinline__ void shmemg_d_putmem(const shmemg_device_ctx_t &c, void *dst, const void *src,
                                                       uint64_t n, int pe) {
    shmemg_d_putmem_group(c, shmemg_d_group_thread(), dst, src, n, pe, shmemg_d_my_pe(c));
}
static __device__ __forceinline__ void shmemg_d_getmem(const shmemg_device_ctx_t &c, void *dst, const void *src,
                                                       uint64_t n, int pe) {
    shmemg_d_getmem_group(c, shmemg_d_group_thread(), dst, src, n, pe, shmemg_d_my_pe(c));
}

/* ------------------------------------------------------------------ ordering (Sec. 6.4) */
/* fence: later RMA/AMO of this thread are ordered after earlier ones (GPU scope). */
static __device__ __forceinline__ void shmemg_d_fence() { shmemg_d_fence_gpu(); }
/* quiet: this thread's earlier plain-store RMA and AMOs are complete and visible at GPU
 * scope.  Host visibility additionally needs the host to synchronise (Fig. 3b). */
static __device__ __forceinline__ void shmemg_d_quiet() { shmemg_d_fence_gpu(); }
/* quiet for a whole PE (all its threads' operations): PE barrier, then a GPU-scope
 * fence by the leader, whose later release covers the PE's writes (cumulativity). */
static __device__ __forceinline__ void shmemg_d_quiet_pe(const shmemg_device_ctx_t &c) {
    shmemg_d_pe_sync(c);
    if (shmemg_d_pe_leader(c)) shmemg_d_fence_gpu();
}

/* ------------------------------------------------------------------ AMOs (Sec. 2.1) */
/* Thread scope, relaxed at GPU scope ("atomicity does not imply ordering", Sec. 6.3). */
static __device__ __forceinline__ int64_t shmemg_d_int64_atomic_fetch_add(const shmemg_device_ctx_t &c,
                                                                          int64_t *target, int64_t v, int pe) {
    return (int64_t)atomicAdd((unsigned long long *)shmemg_d_ptr(c, target, pe), (unsigned long long)v);
}
static __device__ __forceinline__ int64_t shmemg_d_int64_atomic_compare_swap(const shmemg_device_ctx_t &c,
                                                                             int64_t *target, int64_t cond,
                                                                             int64_t v, int pe) {
    return (int64_t)atomicCAS((unsigned long long *)shmemg_d_ptr(c, target, pe), (unsigned long long)cond,
                              (unsigned long long)v);
}
static __device__ __forceinline__ int64_t shmemg_d_int64_atomic_fetch_xor(const shmemg_device_ctx_t &c,
                                                                          int64_t *target, int64_t v, int pe) {
    return (int64_t)atomicXor((unsigned long long *)shmemg_d_ptr(c, target, pe), (unsigned long long)v);
}
static __device__ __forceinline__ int32_t shmemg_d_int32_atomic_fetch_add(const shmemg_device_ctx_t &c,
                                                                          int32_t *target, int32_t v, int pe) {
    return atomicAdd((int *)shmemg_d_ptr(c, target, pe), v);
}
static __device__ __forceinline__ int32_t shmemg_d_int32_atomic_compare_swap(const shmemg_device_ctx_t &c,
                                                                             int32_t *target, int32_t cond,
                                                                             int32_t v, int pe) {
    return atomicCAS((int *)shmemg_d_ptr(c, target, pe), cond, v);
}
static __device__ __forceinline__ int32_t shmemg_d_int32_atomic_fetch_xor(const shmemg_device_ctx_t &c,
                                                                          int32_t *target, int32_t v, int pe) {
    return atomicXor((int *)shmemg_d_ptr(c, target, pe), v);
}

/* ------------------------------------------------------------------ signals */
/* Signal update after the data (Sec. 7, put-signal): release at GPU scope so the data
 * written before it by this thread -- and by the PE's threads synchronised with it --
 * is visible to whoever acquires the signal. */
static __device__ __forceinline__ void shmemg_d_signal_op(uint64_t *sig_addr, uint64_t v, int sig_op) {
    if (sig_op == SHMEMG_SIGNAL_SET) shmemg_d_st_release_u64(sig_addr, v);
    else shmemg_d_red_release_add_u64(sig_addr, v);
}
static __device__ __forceinline__ bool shmemg_d_cmp(uint64_t s, int cmp, uint64_t v) {
    switch (cmp) {
    case SHMEMG_CMP_EQ: return s == v;
    case SHMEMG_CMP_NE: return s != v;
    case SHMEMG_CMP_GT: return s > v;
    case SHMEMG_CMP_GE: return s >= v;
    case SHMEMG_CMP_LT: return s < v;
    default: return s <= v;
    }
}
/* put-with-signal at group scope: the put, a PE-wide completion, then one release
 * update of the signal on `pe` by the group's rank 0. */
static __device__ __forceinline__ void shmemg_d_putmem_signal_block(const shmemg_device_ctx_t &c, void *dst,
                                                                    const void *src, uint64_t n, uint64_t *sig,
                                                                    uint64_t v, int sig_op, int pe) {
    shmemg_d_putmem_group(c, shmemg_d_group_block(), dst, src, n, pe, shmemg_d_my_pe(c));
    __syncthreads();
    if (threadIdx.x == 0) {
        shmemg_d_fence_gpu();
        shmemg_d_signal_op((uint64_t *)shmemg_d_ptr(c, sig, pe), v, sig_op);
    }
    __syncthreads();
}
/* put-with-signal at warp scope: the warp's lanes share the put, lane 0 fences and
 * updates the signal once the warp has written. */
static __device__ __forceinline__ void shmemg_d_putmem_signal_warp(const shmemg_device_ctx_t &c, void *dst,
                                                                   const void *src, uint64_t n, uint64_t *sig,
                                                                   uint64_t v, int sig_op, int pe) {
    shmemg_d_putmem_group(c, shmemg_d_group_warp(), dst, src, n, pe, shmemg_d_my_pe(c));
    __syncwarp();
    if ((threadIdx.x & 31u) == 0) {
        shmemg_d_fence_gpu();
        shmemg_d_signal_op((uint64_t *)shmemg_d_ptr(c, sig, pe), v, sig_op);
    }
    __syncwarp();
}
/* wait_until on the caller's own signal word (thread scope, Sec. 6.4 single unscoped
 * contract), bounded: SHMEMG_SUCCESS or SHMEMG_ERR_TIMEOUT (recorded in the status
 * word with `detail`).  Acquire: data published before the matching release is
 * visible afterwards. */
static __device__ __forceinline__ int shmemg_d_signal_wait_until(const shmemg_device_ctx_t &c, const uint64_t *sig_local,
                                                                 int cmp, uint64_t v, int64_t detail) {
    uint64_t t0 = 0;
    uint32_t ns = 32;
    for (uint32_t it = 0;; it++) {
        if (shmemg_d_cmp(shmemg_d_ld_acquire_u64(sig_local), cmp, v)) return SHMEMG_SUCCESS;
        if ((it & 63) == 0) {
            uint64_t now = shmemg_d_globaltimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > c.timeout_ns) {
                shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, detail);
                return SHMEMG_ERR_TIMEOUT;
            }
            if (shmemg_d_get_status(c) != 0) return SHMEMG_ERR_DEVICE;  /* another PE failed */
        }
        if (it >= 256) {  /* spin first (a signal usually comes within a few round trips), then back off */
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
        }
    }
}

/* ------------------------------------------------------------------ barriers */
/* Barrier of one team group, entered by the leader thread of each member PE after the
 * PE's own quiet.  The slot's count (low half) and generation (high half) form one
 * 64-bit word: a PE arrives with one acq_rel add of 1 (release for the PE's writes,
 * ordered before it by the PE barrier; the old value gives the generation); the last
 * arrival adds 2^32 - size, which resets the count and opens the next generation in one
 * release; the others acquire-poll the word until the generation moves -- spinning at
 * first, then backing off -- bounded.  Needs every member PE resident on the GPU at once. */
static __device__ __forceinline__ int shmemg_d_team_barrier_leader(const shmemg_device_ctx_t &c, int bar_slot,
                                                                   uint32_t size, int64_t detail) {
    shmemg_dbar_t *b = (shmemg_dbar_t *)(c.state + SHMEMG_BARRIERS_OFF) + bar_slot;
    unsigned long long *w = (unsigned long long *)&b->count;  /* count | gen << 32 */
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(w), "l"(1ull) : "memory");
    const uint32_t gen = (uint32_t)(old >> 32);
    if ((uint32_t)old == size - 1) {
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(w), "l"((1ull << 32) - size) : "memory");
        return SHMEMG_SUCCESS;
    }
    uint64_t t0 = 0;
    uint32_t ns = 32;
    for (uint32_t it = 0;; it++) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(w) : "memory");
        if ((uint32_t)(v >> 32) != gen) return SHMEMG_SUCCESS;
        if ((it & 63) == 63) {
            uint64_t now = shmemg_d_globaltimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > c.timeout_ns) {
                shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, detail);
                return SHMEMG_ERR_TIMEOUT;
            }
            if (shmemg_d_get_status(c) != 0) return SHMEMG_ERR_DEVICE;
        }
        if (it >= 256) {  /* a long wait: stop hammering the line */
            __nanosleep(ns);
            if (ns < 512) ns <<= 1;
        }
    }
}

/* ------------------------------------------------------------------ cluster (DSMEM) */
/* The device shared team (Sec. 6.3: the peers that share a GPU memory locality domain)
 * of a CTA-mode heap with cluster_dim > 1 is one hardware thread-block cluster when a
 * kernel is launched with clusters of cluster_dim CTAs: its members can load and store
 * each other's shared memory (distributed shared memory, DSMEM) directly, the direct
 * pointer idea of shmem_ptr (Sec. 4.2) applied to on-chip memory.
 *
 * A kernel using this path keeps one shmemg_cluster_state_t in shared memory and calls
 * shmemg_d_cluster_begin first and shmemg_d_cluster_end last, with every thread of
 * every CTA: a CTA may touch a peer's shared memory only after the peer has started and
 * before it exits, and both calls are hardware cluster barriers.  The shared team's
 * barrier is the hardware cluster barrier too, which has no timeout: such a kernel
 * keeps every CTA of a cluster on the same sequence of cluster barriers, also after an
 * error (a CTA that has failed still passes the barriers of the operations it skips),
 * and every other wait in it is bounded, so every CTA reaches every barrier. */
typedef struct {
    int rc;  /* reserved: the state is what marks a kernel as running the cluster path */
} shmemg_cluster_state_t;

/* Every DSMEM access below names its state space: a peer's copy of a shared-memory
 * object is addressed by its 32-bit shared::cluster address (mapa), the CTA's own copy
 * by its shared::cta address; no generic address points into the cluster window. */
static __device__ __forceinline__ uint32_t shmemg_d_cluster_addr(const void *local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(shmemg_smem_u32(local)), "r"(rank));
    return r;
}
static __device__ __forceinline__ void shmemg_d_st_release_cluster_u64(uint32_t dsm, uint64_t v) {
    asm volatile("st.release.cluster.shared::cluster.u64 [%0], %1;" ::"r"(dsm), "l"(v) : "memory");
}
static __device__ __forceinline__ void shmemg_d_red_release_cluster_add_u64(uint32_t dsm, uint64_t v) {
    asm volatile("red.release.cluster.shared::cluster.add.u64 [%0], %1;" ::"r"(dsm), "l"(v) : "memory");
}
static __device__ __forceinline__ uint64_t shmemg_d_ld_acquire_cluster_u64(const uint64_t *own) {
    uint64_t v;
    asm volatile("ld.acquire.cluster.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(shmemg_smem_u32(own)) : "memory");
    return v;
}
/* plain DSMEM loads and stores of 1, 2, 4, 8 or 16 bytes */
template <int B> struct shmemg_dsm;
template <> struct shmemg_dsm<16> {
    typedef uint4 W;
    static __device__ __forceinline__ W ld(uint32_t a) {
        W v;
        asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "r"(a) : "memory");
        return v;
    }
    static __device__ __forceinline__ void st(uint32_t a, W v) {
        asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z),
                     "r"(v.w) : "memory");
    }
};
template <> struct shmemg_dsm<8> {
    typedef uint2 W;
    static __device__ __forceinline__ W ld(uint32_t a) {
        W v;
        asm volatile("ld.shared::cluster.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
        return v;
    }
    static __device__ __forceinline__ void st(uint32_t a, W v) {
        asm volatile("st.shared::cluster.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(v.x), "r"(v.y) : "memory");
    }
};
template <> struct shmemg_dsm<4> {
    typedef uint32_t W;
    static __device__ __forceinline__ W ld(uint32_t a) {
        W v;
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
        return v;
    }
    static __device__ __forceinline__ void st(uint32_t a, W v) {
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
    }
};
template <> struct shmemg_dsm<2> {
    typedef uint16_t W;
    static __device__ __forceinline__ W ld(uint32_t a) {
        W v;
        asm volatile("ld.shared::cluster.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
        return v;
    }
    static __device__ __forceinline__ void st(uint32_t a, W v) {
        asm volatile("st.shared::cluster.u16 [%0], %1;" ::"r"(a), "h"(v) : "memory");
    }
};
template <> struct shmemg_dsm<1> {
    typedef uint8_t W;
    static __device__ __forceinline__ W ld(uint32_t a) {
        uint32_t v;
        asm volatile("ld.shared::cluster.u8 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
        return (W)v;
    }
    static __device__ __forceinline__ void st(uint32_t a, W v) {
        asm volatile("st.shared::cluster.u8 [%0], %1;" ::"r"(a), "r"((uint32_t)v) : "memory");
    }
};
template <typename V>
static __device__ __forceinline__ V shmemg_d_ld_cluster(uint32_t a) {
    typename shmemg_dsm<sizeof(V)>::W w = shmemg_dsm<sizeof(V)>::ld(a);
    V v;
    memcpy(&v, &w, sizeof(V));
    return v;
}
template <typename V>
static __device__ __forceinline__ void shmemg_d_st_cluster(uint32_t a, V v) {
    typename shmemg_dsm<sizeof(V)>::W w;
    memcpy(&w, &v, sizeof(V));
    shmemg_dsm<sizeof(V)>::st(a, w);
}

static __device__ __forceinline__ void shmemg_d_cluster_begin(shmemg_cluster_state_t &cs) {
    if (threadIdx.x == 0) cs.rc = 0;
    shmemg_d_cluster_sync();
}
static __device__ __forceinline__ void shmemg_d_cluster_end() { shmemg_d_cluster_sync(); }

/* Is `team` the hardware cluster of this launch (its barrier and data can go through
 * DSMEM)?  Only when the kernel keeps a cluster state and the heap's shared team is a
 * cluster of CTAs. */
static __device__ __forceinline__ bool shmemg_d_team_is_cluster(const shmemg_device_ctx_t &c,
                                                                const shmemg_cluster_state_t *cs, int team) {
    return cs && team == SHMEMG_TEAM_SHARED && c.pe_mode == SHMEMG_PE_MODE_CTA && c.cluster_dim > 1;
}

/* Barrier of the cluster's CTAs at CTA scope (every thread of every CTA calls it): the
 * hardware cluster barrier, release/acquire at cluster scope, so that each member sees
 * every write the others made before it.  `quiet` first makes the CTA's earlier writes
 * visible GPU-wide, as a team barrier does.  It cannot fail; the int result keeps the
 * interface of the team barriers. */
static __device__ __forceinline__ int shmemg_d_cluster_sync_pe(const shmemg_device_ctx_t &c,
                                                               shmemg_cluster_state_t &cs, bool quiet, int64_t detail) {
    (void)c;
    (void)cs;
    (void)detail;
    if (quiet) {
        __syncthreads();
        if (threadIdx.x == 0) shmemg_d_fence_gpu();
        __syncwarp();
    }
    shmemg_d_cluster_sync();
    return SHMEMG_SUCCESS;
}

/* Team barrier at PE scope (all threads of the calling PE call it): quiet, then the
 * leader runs the team barrier; the result is broadcast to the PE's threads.  With a
 * cluster state and the cluster's own team, it is the hardware cluster barrier. */
static __device__ __forceinline__ int shmemg_d_team_sync_pe(const shmemg_device_ctx_t &c, int team, int64_t detail,
                                                            shmemg_cluster_state_t *cs = nullptr) {
    if (shmemg_d_team_is_cluster(c, cs, team)) return shmemg_d_cluster_sync_pe(c, *cs, true, detail);
    __shared__ int shmemg_sync_rc;
    const shmemg_dteam_t *t = shmemg_d_team(c, team);
    int grp = 0;
    int r = shmemg_d_team_rank(*t, shmemg_d_my_pe(c), &grp);
    shmemg_d_pe_sync(c);
    if (threadIdx.x == 0) {
        int rc = SHMEMG_SUCCESS;
        if (r >= 0 && shmemg_d_pe_leader(c)) rc = shmemg_d_team_barrier_leader(c, t->bar_base + grp, (uint32_t)t->size, detail);
        shmemg_sync_rc = rc;
    }
    shmemg_d_pe_sync(c);
    /* in pe_mode CLUSTER every CTA takes the leader CTA's result, read through DSMEM, so
     * the CTAs of a PE decide as one (their hardware PE barriers stay in step); the
     * leader writes the slot again only after the next PE barrier, which every CTA
     * reaches after this read */
    if (c.pe_mode == SHMEMG_PE_MODE_CLUSTER && c.cluster_dim > 1)
        return shmemg_d_ld_cluster<int>(shmemg_d_cluster_addr(&shmemg_sync_rc, 0));
    return shmemg_sync_rc;
}
static __device__ __forceinline__ int shmemg_d_barrier_all_pe(const shmemg_device_ctx_t &c, int64_t detail) {
    return shmemg_d_team_sync_pe(c, SHMEMG_TEAM_WORLD, detail);
}


/* ------------------------------------------------------------------ reductions */

template <typename V> struct shmemg_vadd;
template <> struct shmemg_vadd<float4> {
    static __device__ __forceinline__ float4 add(float4 a, float4 b) {
        return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
    }
};
template <> struct shmemg_vadd<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
};

/* Sum of member values over the aligned rank block [r0, r0 + 2^L), by recursive
 * halving: the rank-pairwise tree restricted to that block. */
template <int L, typename V>
static __device__ __forceinline__ V shmemg_tree_block(const uint8_t *heap, uint64_t H, int pe0, int pstride, int r0,
                                                      uint64_t off) {
    if constexpr (L == 0) {
        return shmemg_ld_cg((const V *)(heap + (uint64_t)(pe0 + r0 * pstride) * H + off));
    } else {
        V a = shmemg_tree_block<L - 1, V>(heap, H, pe0, pstride, r0, off);
        V b = shmemg_tree_block<L - 1, V>(heap, H, pe0, pstride, r0 + (1 << (L - 1)), off);
        return shmemg_vadd<V>::add(a, b);
    }
}

/* Fixed float reduction order: the rank-pairwise tree over P members (level by level,
 * pairs (2i, 2i+1), an odd last value carried up).  It equals the sum of the aligned
 * power-of-two rank blocks of P's binary expansion, combined from the right, which is
 * how it is evaluated here (bitwise identical, order fixed for every P).  Blocks of up to
 * 2^MAXB ranks are unrolled (2^MAXB loads in flight per thread); a larger block is the
 * pairwise tree over its 2^MAXB-rank sub-blocks, combined with a carry stack (a binary
 * counter), which is the same pairing. */
template <typename V, int MAXB = 5>
static __device__ __forceinline__ V shmemg_tree_sum(const uint8_t *heap, uint64_t H, int pe0, int pstride, int P,
                                                    uint64_t off) {
    static_assert(MAXB >= 1 && MAXB <= 5, "unrolled block size");
    V acc{};
    bool have = false;
#define SHMEMG_TB(b)                                                                         \
    if constexpr (b <= MAXB) {                                                               \
        if (P & (1 << b)) {                                                                  \
            V t = shmemg_tree_block<b, V>(heap, H, pe0, pstride, P & ~((2 << b) - 1), off);  \
            acc = have ? shmemg_vadd<V>::add(t, acc) : t;                                    \
            have = true;                                                                     \
        }                                                                                    \
    }
    SHMEMG_TB(0) SHMEMG_TB(1) SHMEMG_TB(2) SHMEMG_TB(3) SHMEMG_TB(4) SHMEMG_TB(5)
#undef SHMEMG_TB
    for (int b = MAXB + 1; b < 31; b++) {
        if (!(P & (1 << b))) continue;
        int s0 = P & ~((2 << b) - 1);
        int nsub = 1 << (b - MAXB);
        V stack[31 - MAXB];
        V v{};
        for (int q = 0; q < nsub; q++) {
            v = shmemg_tree_block<MAXB, V>(heap, H, pe0, pstride, s0 + (q << MAXB), off);
            int cnt = q, j = 0;
            while (cnt & 1) {
                v = shmemg_vadd<V>::add(stack[j], v);
                cnt >>= 1;
                j++;
            }
            stack[j] = v;
        }
        acc = have ? shmemg_vadd<V>::add(v, acc) : v;
        have = true;
    }
    return acc;
}

template <typename T> static __device__ __forceinline__ T shmemg_comb(T a, T b, int op);
template <> __device__ __forceinline__ int32_t shmemg_comb<int32_t>(int32_t a, int32_t b, int op) {
    return op == SHMEMG_SUM ? (int32_t)((uint32_t)a + (uint32_t)b) : op == SHMEMG_MAX ? max(a, b) : min(a, b);
}
template <> __device__ __forceinline__ int64_t shmemg_comb<int64_t>(int64_t a, int64_t b, int op) {
    return op == SHMEMG_SUM ? (int64_t)((uint64_t)a + (uint64_t)b) : op == SHMEMG_MAX ? max(a, b) : min(a, b);
}
template <> __device__ __forceinline__ float shmemg_comb<float>(float a, float b, int op) {
    return op == SHMEMG_MAX ? (b > a ? b : a) : (b < a ? b : a);  /* sums use the tree */
}

/* Slice-owner reduce of vectors [v0, v1) (V = T or a 16-byte vector of T): each thread
 * of g owns vectors, reads them from the P members pe0 + r*pstride, combines (integer
 * sums wrap; float sums by the rank-pairwise tree; max/min exact) and writes the result
 * to every member's dst. */
template <typename T, typename V, int OP, int TREE_MAXB = 5>
static __device__ __forceinline__ void shmemg_d_reduce_vecs(shmemg_group g, uint8_t *heap, uint64_t H, int pe0,
                                                           int pstride, int P, uint64_t dst_off, uint64_t src_off,
                                                           uint64_t v0, uint64_t v1) {
    constexpr int NL = sizeof(V) / sizeof(T);
    for (uint64_t vi = v0 + g.rank; vi < v1; vi += g.size) {
        const uint64_t off = src_off + vi * sizeof(V);
        V acc;
        if constexpr (OP == SHMEMG_SUM && std::is_floating_point<T>::value) {
            acc = shmemg_tree_sum<V, TREE_MAXB>(heap, H, pe0, pstride, P, off);
        } else {
            acc = shmemg_ld_cg((const V *)(heap + (uint64_t)pe0 * H + off));
            int r = 1;
            for (; r + 7 < P; r += 8) {  /* eight members' loads in flight */
                V x[8];
#pragma unroll
                for (int u = 0; u < 8; u++) x[u] = shmemg_ld_cg((const V *)(heap + (uint64_t)(pe0 + (r + u) * pstride) * H + off));
#pragma unroll
                for (int u = 0; u < 8; u++)
#pragma unroll
                    for (int l = 0; l < NL; l++) {
                        T &s = reinterpret_cast<T *>(&acc)[l];
                        s = shmemg_comb<T>(s, reinterpret_cast<T *>(&x[u])[l], OP);
                    }
            }
            for (; r + 3 < P; r += 4) {
                V a = shmemg_ld_cg((const V *)(heap + (uint64_t)(pe0 + r * pstride) * H + off));
                V b = shmemg_ld_cg((const V *)(heap + (uint64_t)(pe0 + (r + 1) * pstride) * H + off));
                V d = shmemg_ld_cg((const V *)(heap + (uint64_t)(pe0 + (r + 2) * pstride) * H + off));
                V e = shmemg_ld_cg((const V *)(heap + (uint64_t)(pe0 + (r + 3) * pstride) * H + off));
#pragma unroll
                for (int l = 0; l < NL; l++) {
                    T &s = reinterpret_cast<T *>(&acc)[l];
                    s = shmemg_comb<T>(s, reinterpret_cast<T *>(&a)[l], OP);
                    s = shmemg_comb<T>(s, reinterpret_cast<T *>(&b)[l], OP);
                    s = shmemg_comb<T>(s, reinterpret_cast<T *>(&d)[l], OP);
                    s = shmemg_comb<T>(s, reinterpret_cast<T *>(&e)[l], OP);
                }
            }
            for (; r < P; r++) {
                V a = shmemg_ld_cg((const V *)(heap + (uint64_t)(pe0 + r * pstride) * H + off));
#pragma unroll
                for (int l = 0; l < NL; l++) {
                    T &s = reinterpret_cast<T *>(&acc)[l];
                    s = shmemg_comb<T>(s, reinterpret_cast<T *>(&a)[l], OP);
                }
            }
        }
        const uint64_t doff = dst_off + vi * sizeof(V);
        for (int r = 0; r < P; r++) *(V *)(heap + (uint64_t)(pe0 + r * pstride) * H + doff) = acc;
    }
}

/* dispatch on element type, op and vector width (16-byte vectors when every address
 * and the element range allow it); TREE_MAXB bounds the float tree's unrolled blocks */
template <typename T, typename V16, int TREE_MAXB = 5>
static __device__ __forceinline__ void shmemg_d_reduce_elems_t(shmemg_group g, uint8_t *heap, uint64_t H, int pe0,
                                                              int pstride, int P, uint64_t dst_off, uint64_t src_off,
                                                              uint64_t e0, uint64_t e1, int op) {
    constexpr uint64_t L = sizeof(V16) / sizeof(T);
    const bool v16 = ((dst_off | src_off | (e0 * sizeof(T)) | (e1 * sizeof(T)) | H) & 15) == 0;
    if (v16) {
        if (op == SHMEMG_SUM) shmemg_d_reduce_vecs<T, V16, SHMEMG_SUM, TREE_MAXB>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0 / L, e1 / L);
        else if (op == SHMEMG_MAX) shmemg_d_reduce_vecs<T, V16, SHMEMG_MAX>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0 / L, e1 / L);
        else shmemg_d_reduce_vecs<T, V16, SHMEMG_MIN>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0 / L, e1 / L);
    } else {
        if (op == SHMEMG_SUM) shmemg_d_reduce_vecs<T, T, SHMEMG_SUM, TREE_MAXB>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0, e1);
        else if (op == SHMEMG_MAX) shmemg_d_reduce_vecs<T, T, SHMEMG_MAX>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0, e1);
        else shmemg_d_reduce_vecs<T, T, SHMEMG_MIN>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0, e1);
    }
}
static __device__ __forceinline__ void shmemg_d_reduce_elems(shmemg_group g, uint8_t *heap, uint64_t H, int pe0,
                                                            int pstride, int P, uint64_t dst_off, uint64_t src_off,
                                                            uint64_t e0, uint64_t e1, int dtype, int op) {
    if (dtype == SHMEMG_INT32) shmemg_d_reduce_elems_t<int32_t, int4>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0, e1, op);
    else if (dtype == SHMEMG_INT64) shmemg_d_reduce_elems_t<int64_t, longlong2>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0, e1, op);
    else shmemg_d_reduce_elems_t<float, float4>(g, heap, H, pe0, pstride, P, dst_off, src_off, e0, e1, op);
}

/* Group-wide copy of src to the same offset `dst_off` of P members (one read, P
 * writes per vector). */
template <typename V>
static __device__ __forceinline__ void shmemg_d_replicate_vec(shmemg_group g, uint8_t *heap, uint64_t H, int pe0,
                                                             int pstride, int P, uint64_t dst_off, const V *src,
                                                             uint64_t v0, uint64_t v1) {
    for (uint64_t vi = v0 + g.rank; vi < v1; vi += g.size) {
        V a = shmemg_ld_cg(src + vi);
        for (int r = 0; r < P; r++) ((V *)(heap + (uint64_t)(pe0 + r * pstride) * H + dst_off))[vi] = a;
    }
}
/* bytes [b0, b1) of src -> the same bytes of dst_off on every member */
static __device__ __forceinline__ void shmemg_d_replicate_bytes(shmemg_group g, uint8_t *heap, uint64_t H, int pe0,
                                                               int pstride, int P, uint64_t dst_off, const uint8_t *src,
                                                               uint64_t b0, uint64_t b1) {
    const int w = shmemg_d_vec_width((const void *)(heap + dst_off), src, b0 | b1 | H);
    switch (w) {
    case 16: shmemg_d_replicate_vec(g, heap, H, pe0, pstride, P, dst_off, (const uint4 *)src, b0 / 16, b1 / 16); break;
    case 8: shmemg_d_replicate_vec(g, heap, H, pe0, pstride, P, dst_off, (const uint2 *)src, b0 / 8, b1 / 8); break;
    case 4: shmemg_d_replicate_vec(g, heap, H, pe0, pstride, P, dst_off, (const uint32_t *)src, b0 / 4, b1 / 4); break;
    case 2: shmemg_d_replicate_vec(g, heap, H, pe0, pstride, P, dst_off, (const uint16_t *)src, b0 / 2, b1 / 2); break;
    default: shmemg_d_replicate_vec(g, heap, H, pe0, pstride, P, dst_off, (const uint8_t *)src, b0, b1); break;
    }
}

/* slice [lo, hi) of `total` units owned by rank r of P, in multiples of `gran` units */
static __device__ __forceinline__ void shmemg_d_slice(uint64_t total, int r, int P, uint64_t gran, uint64_t *lo,
                                                      uint64_t *hi) {
    uint64_t blocks = (total + gran - 1) / gran;
    uint64_t b0 = blocks * (uint64_t)r / (uint64_t)P, b1 = blocks * (uint64_t)(r + 1) / (uint64_t)P;
    *lo = b0 * gran < total ? b0 * gran : total;
    *hi = b1 * gran < total ? b1 * gran : total;
}

/* ------------------------------------------------------------------ device collectives */
/* Warp-scope team barrier (Sec. 6.3 participation scopes: one warp of the PE calls it,
 * all 32 lanes with identical arguments): lane 0 quiets the warp's writes and runs the
 * team barrier for the PE; the result is broadcast to the warp. */
static __device__ __forceinline__ int shmemg_d_team_sync_warp(const shmemg_device_ctx_t &c, int team, int64_t detail) {
    const shmemg_dteam_t *t = shmemg_d_team(c, team);
    int grp = 0;
    const int r = shmemg_d_team_rank(*t, shmemg_d_my_pe(c), &grp);
    __syncwarp();
    int rc = SHMEMG_SUCCESS;
    if ((threadIdx.x & 31u) == 0 && r >= 0)
        rc = shmemg_d_team_barrier_leader(c, t->bar_base + grp, (uint32_t)t->size, detail);
    rc = __shfl_sync(0xffffffffu, rc, 0);
    __syncwarp();
    return rc;
}

/* Participation scope of a device collective: the threads that cooperate and the team
 * synchronisation they use.  PE scope: every thread of the PE (its block, or its
 * cluster in pe_mode CLUSTER); warp scope: one warp of the PE.  A runtime choice, so
 * both scopes share one copy of the data-movement code. */
static __device__ __forceinline__ shmemg_group shmemg_d_scope_group(const shmemg_device_ctx_t &c, bool warp) {
    return warp ? shmemg_d_group_warp() : shmemg_d_group_pe(c);
}
static __device__ __forceinline__ int shmemg_d_scope_sync(const shmemg_device_ctx_t &c, int team, int64_t detail,
                                                          shmemg_cluster_state_t *cs, bool warp) {
    return warp ? shmemg_d_team_sync_warp(c, team, detail) : shmemg_d_team_sync_pe(c, team, detail, cs);
}

/* Team collectives at PE or warp scope (every participating thread of every member PE
 * calls with identical arguments: Sec. 6.3 uniform participation).  Each quiets and
 * synchronises the team on entry and exit; in between, member r does its share: a
 * slice of the elements or bytes (reduce, broadcast) or its own blocks (fcollect,
 * alltoall).  Offsets are symmetric byte offsets.  Return SHMEMG_SUCCESS or a timeout /
 * device error. */
static __device__ __forceinline__ int shmemg_d_reduce_scoped(const shmemg_device_ctx_t &c, int team, uint64_t dst_off,
                                                             uint64_t src_off, uint64_t nelems, int dtype, int op,
                                                             int64_t detail, shmemg_cluster_state_t *cs, bool warp) {
    const shmemg_dteam_t t = *shmemg_d_team(c, team);
    int grp = 0, r = shmemg_d_team_rank(t, shmemg_d_my_pe(c), &grp);
    if (r < 0) return SHMEMG_SUCCESS;
    int rc = shmemg_d_scope_sync(c, team, detail, cs, warp);
    if (rc) return rc;
    uint64_t es = dtype == SHMEMG_INT64 ? 8 : 4, lo, hi;
    shmemg_d_slice(nelems, r, t.size, 16 / es, &lo, &hi);
    shmemg_d_reduce_elems(shmemg_d_scope_group(c, warp), c.heap, c.pe_stride, shmemg_d_team_member(t, grp, 0),
                          t.stride, t.size, dst_off, src_off, lo, hi, dtype, op);
    return shmemg_d_scope_sync(c, team, detail, cs, warp);
}
static __device__ __forceinline__ int shmemg_d_broadcastmem_scoped(const shmemg_device_ctx_t &c, int team,
                                                                   uint64_t dst_off, uint64_t src_off, uint64_t n,
                                                                   int root, int64_t detail, shmemg_cluster_state_t *cs,
                                                                   bool warp) {
    const shmemg_dteam_t t = *shmemg_d_team(c, team);
    int grp = 0, r = shmemg_d_team_rank(t, shmemg_d_my_pe(c), &grp);
    if (r < 0) return SHMEMG_SUCCESS;
    int rc = shmemg_d_scope_sync(c, team, detail, cs, warp);
    if (rc) return rc;
    uint64_t lo, hi;
    shmemg_d_slice(n, r, t.size, 16, &lo, &hi);
    const uint8_t *src = shmemg_d_addr(c, shmemg_d_team_member(t, grp, root), src_off);
    shmemg_d_replicate_bytes(shmemg_d_scope_group(c, warp), c.heap, c.pe_stride, shmemg_d_team_member(t, grp, 0),
                             t.stride, t.size, dst_off, src, lo, hi);
    return shmemg_d_scope_sync(c, team, detail, cs, warp);
}
static __device__ __forceinline__ int shmemg_d_fcollectmem_scoped(const shmemg_device_ctx_t &c, int team,
                                                                  uint64_t dst_off, uint64_t src_off, uint64_t n,
                                                                  int64_t detail, shmemg_cluster_state_t *cs, bool warp) {
    const shmemg_dteam_t t = *shmemg_d_team(c, team);
    int grp = 0, r = shmemg_d_team_rank(t, shmemg_d_my_pe(c), &grp);
    if (r < 0) return SHMEMG_SUCCESS;
    int rc = shmemg_d_scope_sync(c, team, detail, cs, warp);
    if (rc) return rc;
    const uint8_t *src = shmemg_d_addr(c, shmemg_d_team_member(t, grp, r), src_off);
    shmemg_d_replicate_bytes(shmemg_d_scope_group(c, warp), c.heap, c.pe_stride, shmemg_d_team_member(t, grp, 0),
                             t.stride, t.size, dst_off + (uint64_t)r * n, src, 0, n);
    return shmemg_d_scope_sync(c, team, detail, cs, warp);
}
static __device__ __forceinline__ int shmemg_d_alltoallmem_scoped(const shmemg_device_ctx_t &c, int team,
                                                                  uint64_t dst_off, uint64_t src_off, uint64_t n,
                                                                  int64_t detail, shmemg_cluster_state_t *cs, bool warp) {
    const shmemg_dteam_t t = *shmemg_d_team(c, team);
    int grp = 0, r = shmemg_d_team_rank(t, shmemg_d_my_pe(c), &grp);
    if (r < 0) return SHMEMG_SUCCESS;
    int rc = shmemg_d_scope_sync(c, team, detail, cs, warp);
    if (rc) return rc;
    const int me = shmemg_d_team_member(t, grp, r);
    for (int j = 0; j < t.size; j++) {
        int pj = shmemg_d_team_member(t, grp, j);
        shmemg_d_copy_group(shmemg_d_scope_group(c, warp), shmemg_d_addr(c, pj, dst_off + (uint64_t)r * n),
                            shmemg_d_addr(c, me, src_off + (uint64_t)j * n), n);
    }
    return shmemg_d_scope_sync(c, team, detail, cs, warp);
}

/* PE scope: every thread of the PE; with a cluster state, the shared team's barrier is
 * the hardware cluster barrier */
static __device__ __forceinline__ int shmemg_d_reduce_pe(const shmemg_device_ctx_t &c, int team, uint64_t dst_off,
                                                         uint64_t src_off, uint64_t nelems, int dtype, int op,
                                                         int64_t detail, shmemg_cluster_state_t *cs = nullptr) {
    return shmemg_d_reduce_scoped(c, team, dst_off, src_off, nelems, dtype, op, detail, cs, false);
}
static __device__ __forceinline__ int shmemg_d_broadcastmem_pe(const shmemg_device_ctx_t &c, int team, uint64_t dst_off,
                                                               uint64_t src_off, uint64_t n, int root, int64_t detail,
                                                               shmemg_cluster_state_t *cs = nullptr) {
    return shmemg_d_broadcastmem_scoped(c, team, dst_off, src_off, n, root, detail, cs, false);
}
static __device__ __forceinline__ int shmemg_d_fcollectmem_pe(const shmemg_device_ctx_t &c, int team, uint64_t dst_off,
                                                              uint64_t src_off, uint64_t n, int64_t detail,
                                                              shmemg_cluster_state_t *cs = nullptr) {
    return shmemg_d_fcollectmem_scoped(c, team, dst_off, src_off, n, detail, cs, false);
}
static __device__ __forceinline__ int shmemg_d_alltoallmem_pe(const shmemg_device_ctx_t &c, int team, uint64_t dst_off,
                                                              uint64_t src_off, uint64_t n, int64_t detail,
                                                              shmemg_cluster_state_t *cs = nullptr) {
    return shmemg_d_alltoallmem_scoped(c, team, dst_off, src_off, n, detail, cs, false);
}
/* warp scope: one warp of each member PE (all 32 lanes) */
static __device__ __forceinline__ int shmemg_d_reduce_warp(const shmemg_device_ctx_t &c, int team, uint64_t dst_off,
                                                           uint64_t src_off, uint64_t nelems, int dtype, int op,
                                                           int64_t detail) {
    return shmemg_d_reduce_scoped(c, team, dst_off, src_off, nelems, dtype, op, detail, nullptr, true);
}
static __device__ __forceinline__ int shmemg_d_broadcastmem_warp(const shmemg_device_ctx_t &c, int team,
                                                                 uint64_t dst_off, uint64_t src_off, uint64_t n,
                                                                 int root, int64_t detail) {
    return shmemg_d_broadcastmem_scoped(c, team, dst_off, src_off, n, root, detail, nullptr, true);
}
static __device__ __forceinline__ int shmemg_d_fcollectmem_warp(const shmemg_device_ctx_t &c, int team,
                                                                uint64_t dst_off, uint64_t src_off, uint64_t n,
                                                                int64_t detail) {
    return shmemg_d_fcollectmem_scoped(c, team, dst_off, src_off, n, detail, nullptr, true);
}
static __device__ __forceinline__ int shmemg_d_alltoallmem_warp(const shmemg_device_ctx_t &c, int team,
                                                                uint64_t dst_off, uint64_t src_off, uint64_t n,
                                                                int64_t detail) {
    return shmemg_d_alltoallmem_scoped(c, team, dst_off, src_off, n, detail, nullptr, true);
}

/* ------------------------------------------------------------------ cluster collectives */
/* Shared-team alltoall staged through DSMEM (CTA-mode heaps, the team = the launch's
 * cluster).  `win` is a shared-memory window at the same offset in every CTA (16-byte
 * aligned).  After the entry barrier (a quiet and a team barrier) each member copies its
 * P blocks into its own window, the cluster synchronises, and each member builds ITS OWN
 * destination from the members' windows read through DSMEM; an exit barrier keeps every
 * window until all have read it.  The only HBM traffic is each member's own source read
 * and destination write.  Staging pays for small blocks only: it copies every byte twice
 * and takes a third cluster barrier, so the other shared-team collectives (and larger
 * alltoalls) move their data through L2 between two cluster barriers. */

/* group-wide copies between global memory and a cluster peer's shared memory: the
 * peer's copy of the shared object at `local` in cluster rank `rank` */
template <typename V>
static __device__ __forceinline__ void shmemg_d_copy_vec_from_cluster(shmemg_group g, V *dst, uint32_t src,
                                                                     uint64_t nvec) {
    uint64_t i = g.rank;
    const uint64_t s = g.size;
    for (; i + 3 * s < nvec; i += 4 * s) {
        V a = shmemg_d_ld_cluster<V>(src + (uint32_t)(i * sizeof(V)));
        V b = shmemg_d_ld_cluster<V>(src + (uint32_t)((i + s) * sizeof(V)));
        V d = shmemg_d_ld_cluster<V>(src + (uint32_t)((i + 2 * s) * sizeof(V)));
        V e = shmemg_d_ld_cluster<V>(src + (uint32_t)((i + 3 * s) * sizeof(V)));
        dst[i] = a;
        dst[i + s] = b;
        dst[i + 2 * s] = d;
        dst[i + 3 * s] = e;
    }
    for (; i < nvec; i += s) dst[i] = shmemg_d_ld_cluster<V>(src + (uint32_t)(i * sizeof(V)));
}
static __device__ __forceinline__ void shmemg_d_copy_from_cluster(shmemg_group g, void *dst, const void *local,
                                                                 uint32_t rank, uint64_t n) {
    const uint32_t a = shmemg_d_cluster_addr(local, rank);
    switch (shmemg_d_vec_width(dst, local, n)) {
    case 16: shmemg_d_copy_vec_from_cluster(g, (uint4 *)dst, a, n / 16); break;
    case 8: shmemg_d_copy_vec_from_cluster(g, (uint2 *)dst, a, n / 8); break;
    case 4: shmemg_d_copy_vec_from_cluster(g, (uint32_t *)dst, a, n / 4); break;
    case 2: shmemg_d_copy_vec_from_cluster(g, (uint16_t *)dst, a, n / 2); break;
    default: shmemg_d_copy_vec_from_cluster(g, (uint8_t *)dst, a, n); break;
    }
}
template <typename V>
static __device__ __forceinline__ void shmemg_d_copy_vec_to_cluster(shmemg_group g, uint32_t dst, const V *src,
                                                                   uint64_t nvec) {
    uint64_t i = g.rank;
    const uint64_t s = g.size;
    for (; i + 3 * s < nvec; i += 4 * s) {
        V a = shmemg_ld_cg(src + i), b = shmemg_ld_cg(src + i + s);
        V d = shmemg_ld_cg(src + i + 2 * s), e = shmemg_ld_cg(src + i + 3 * s);
        shmemg_d_st_cluster<V>(dst + (uint32_t)(i * sizeof(V)), a);
        shmemg_d_st_cluster<V>(dst + (uint32_t)((i + s) * sizeof(V)), b);
        shmemg_d_st_cluster<V>(dst + (uint32_t)((i + 2 * s) * sizeof(V)), d);
        shmemg_d_st_cluster<V>(dst + (uint32_t)((i + 3 * s) * sizeof(V)), e);
    }
    for (; i < nvec; i += s) shmemg_d_st_cluster<V>(dst + (uint32_t)(i * sizeof(V)), shmemg_ld_cg(src + i));
}
static __device__ __forceinline__ void shmemg_d_copy_to_cluster(shmemg_group g, void *local, uint32_t rank,
                                                               const void *src, uint64_t n) {
    const uint32_t a = shmemg_d_cluster_addr(local, rank);
    switch (shmemg_d_vec_width(local, src, n)) {
    case 16: shmemg_d_copy_vec_to_cluster(g, a, (const uint4 *)src, n / 16); break;
    case 8: shmemg_d_copy_vec_to_cluster(g, a, (const uint2 *)src, n / 8); break;
    case 4: shmemg_d_copy_vec_to_cluster(g, a, (const uint32_t *)src, n / 4); break;
    case 2: shmemg_d_copy_vec_to_cluster(g, a, (const uint16_t *)src, n / 2); break;
    default: shmemg_d_copy_vec_to_cluster(g, a, (const uint8_t *)src, n); break;
    }
}

/* Gather of nj blocks of nv vectors: block b (rank j0 + b) of the members' windows at
 * byte offset woff -> dst + b * blk.  Four blocks' loads are in flight per thread. */
template <typename V>
static __device__ __forceinline__ void shmemg_d_cluster_gather_vec(uint8_t *dst, uint64_t blk, const uint8_t *win,
                                                                  uint64_t woff, int j0, int nj, uint64_t nv) {
    const uint32_t w0 = shmemg_d_cluster_addr(win, 0);
    const uint32_t wstride = shmemg_d_cluster_addr(win, 1) - w0;
    const uint64_t total = nv * (uint64_t)nj, step = blockDim.x;
    auto src = [&](uint64_t k, uint64_t *b, uint64_t *i) {
        *b = k / nv;
        *i = k - *b * nv;
        return w0 + (uint32_t)(j0 + *b) * wstride + (uint32_t)(woff + *i * sizeof(V));
    };
    uint64_t k = threadIdx.x;
    for (; k + 3 * step < total; k += 4 * step) {
        uint64_t b[4], i[4];
        V x[4];
#pragma unroll
        for (int u = 0; u < 4; u++) x[u] = shmemg_d_ld_cluster<V>(src(k + u * step, &b[u], &i[u]));
#pragma unroll
        for (int u = 0; u < 4; u++) *(V *)(dst + b[u] * blk + i[u] * sizeof(V)) = x[u];
    }
    for (; k < total; k += step) {
        uint64_t b, i;
        const V x = shmemg_d_ld_cluster<V>(src(k, &b, &i));
        *(V *)(dst + b * blk + i * sizeof(V)) = x;
    }
}
static __device__ __forceinline__ void shmemg_d_cluster_gather(uint8_t *dst, uint64_t n, const uint8_t *win,
                                                              uint64_t woff, int j0, int nj) {
    switch (shmemg_d_vec_width(dst, win + woff, n)) {
    case 16: shmemg_d_cluster_gather_vec<uint4>(dst, n, win, woff, j0, nj, n / 16); break;
    case 8: shmemg_d_cluster_gather_vec<uint2>(dst, n, win, woff, j0, nj, n / 8); break;
    case 4: shmemg_d_cluster_gather_vec<uint32_t>(dst, n, win, woff, j0, nj, n / 4); break;
    case 2: shmemg_d_cluster_gather_vec<uint16_t>(dst, n, win, woff, j0, nj, n / 2); break;
    default: shmemg_d_cluster_gather_vec<uint8_t>(dst, n, win, woff, j0, nj, n); break;
    }
}

/* each member stages its P blocks; member r's dst block j = block r of member j's window */
static __device__ __noinline__ int shmemg_d_cluster_alltoallmem_pe(const shmemg_device_ctx_t &c,
                                                                   shmemg_cluster_state_t &cs, uint8_t *win,
                                                                   uint64_t dst_off, uint64_t src_off, uint64_t n,
                                                                   int64_t detail) {
    const int me = shmemg_d_my_pe(c), P = (int)shmemg_d_cluster_nctarank(), r = (int)shmemg_d_cluster_ctarank();
    int rc = shmemg_d_cluster_sync_pe(c, cs, true, detail);
    if (rc) return rc;
    shmemg_d_copy_group(shmemg_d_group_block(), win, shmemg_d_addr(c, me, src_off), n * (uint64_t)P);
    if ((rc = shmemg_d_cluster_sync_pe(c, cs, false, detail))) return rc;
    shmemg_d_cluster_gather(shmemg_d_addr(c, me, dst_off), n, win, (uint64_t)r * n, 0, P);
    return shmemg_d_cluster_sync_pe(c, cs, false, detail);
}

/* put-with-signal into a cluster peer's shared memory (group scope: every thread of g
 * calls; g's rank-0 thread updates the signal after the group has written): n bytes
 * from `src` (global memory) to the peer's copy of the shared object `dst_local`,
 * then a cluster-scope release update of the peer's copy of `sig_local`. */
static __device__ __forceinline__ void shmemg_d_putmem_signal_cluster_block(void *dst_local, const void *src, uint64_t n,
                                                                            uint64_t *sig_local, uint64_t v, int sig_op,
                                                                            uint32_t peer_rank) {
    shmemg_d_copy_to_cluster(shmemg_d_group_block(), dst_local, peer_rank, src, n);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t s = shmemg_d_cluster_addr(sig_local, peer_rank);
        if (sig_op == SHMEMG_SIGNAL_SET) shmemg_d_st_release_cluster_u64(s, v);
        else shmemg_d_red_release_cluster_add_u64(s, v);
    }
}
/* wait_until on the caller's own shared-memory signal word (thread scope, acquire at
 * cluster scope), bounded like shmemg_d_signal_wait_until. */
static __device__ __forceinline__ int shmemg_d_signal_wait_until_cluster(const shmemg_device_ctx_t &c,
                                                                         const uint64_t *sig_local, int cmp, uint64_t v,
                                                                         int64_t detail) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; it++) {
        if (shmemg_d_cmp(shmemg_d_ld_acquire_cluster_u64(sig_local), cmp, v)) return SHMEMG_SUCCESS;
        if ((it & 255) == 255) {
            const uint64_t now = shmemg_d_globaltimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > c.timeout_ns) {
                shmemg_d_set_status(c, SHMEMG_ERR_TIMEOUT, detail);
                return SHMEMG_ERR_TIMEOUT;
            }
            if (shmemg_d_get_status(c) != 0) return SHMEMG_ERR_DEVICE;
        }
    }
}

#endif /* SHMEMG_DEVICE_CUH */
