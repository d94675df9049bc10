// Device-initiated AMO stress stream and put-with-signal ping-pong (paper Sec. 2.1
// atomics; Sec. 6.3 "atomicity does not imply ordering"; Sec. 7 put-signal; case
// study 2 of Sec. 4.4: fine-grained atomics and polling flags in graph analytics).
#include <cuda_runtime.h>

#include "internal.h"

namespace shmemg {

constexpr int AMO_THREADS = 256;
constexpr int PP_THREADS = 128;

// splitmix64 (Steele, Lea, Flood, OOPSLA 2014): first output of the stream seeded with
// seed ^ i -- the counter-based draw both the kernel and the host generators use.
__device__ __forceinline__ uint64_t cb64(uint64_t seed, uint64_t i) {
    uint64_t z = (seed ^ i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct AmoArgs {
    uint8_t *heap;
    uint64_t H;
    uint64_t table_off;   // symmetric offset of the table
    uint64_t wpp;         // words per PE
    int wpp_log2;         // log2(wpp) when a power of two, else -1
    int npes;
    const uint32_t *ops;
    uint64_t nops;
    uint64_t op_seed, table_seed;
    int64_t *fetched;
    uint32_t flags;
    uint64_t nwords;      // npes * wpp
    uint8_t *state;       // reserved prefix (status word)
};

// One CTA per PE; PE p issues ops [p*nops/npes, (p+1)*nops/npes), a warp handles 32
// consecutive ops per iteration (coalesced op reads and fetched writes).
__global__ void __launch_bounds__(AMO_THREADS) k_amo_stream(AmoArgs a) {
    __shared__ uint64_t s_val[AMO_THREADS];
    __shared__ uint64_t s_old[AMO_THREADS];
    const int p = blockIdx.x;
    const uint64_t lo = a.nops * (uint64_t)p / (uint64_t)a.npes;
    const uint64_t hi = a.nops * (uint64_t)(p + 1) / (uint64_t)a.npes;
    if (!(a.flags & SHMEMG_AMO_AGGREGATE)) {
        // each thread keeps four independent atomics in flight (ops i, i+B, i+2B, i+3B)
        constexpr int U = 4;
        for (uint64_t base = lo + threadIdx.x; base < hi; base += (uint64_t)blockDim.x * U) {
            unsigned long long old[U];
            bool act[U];
#pragma unroll
            for (int k = 0; k < U; k++) {
                const uint64_t i = base + (uint64_t)k * blockDim.x;
                act[k] = i < hi;
                old[k] = 0;
                if (!act[k]) continue;
                const uint32_t op = __ldcs(a.ops + i);
                const uint64_t w = op & ((1u << 27) - 1u);
                const uint32_t code = (op >> 27) & 3u;
                if (w >= a.nwords || code == 3u) {
                    int *stw = (int *)(a.state + SHMEMG_STATUS_OFF);
                    if (atomicCAS(stw, 0, SHMEMG_ERR_INVALID_ARG) == 0) *(volatile int64_t *)(a.state + SHMEMG_STATUS_OFF + 8) = (int64_t)i;
                    act[k] = false;
                    continue;
                }
                const uint64_t r = cb64(a.op_seed, i);
                const uint64_t pe = a.wpp_log2 >= 0 ? w >> a.wpp_log2 : w / a.wpp;
                const uint64_t idx = w - pe * a.wpp;
                unsigned long long *addr = (unsigned long long *)(a.heap + pe * a.H + a.table_off + idx * 8);
                if (code == 1u) old[k] = atomicCAS(addr, (unsigned long long)cb64(a.table_seed, w), (unsigned long long)r);
                else if (code == 0u) old[k] = atomicAdd(addr, (unsigned long long)((r & ((1u << 20) - 1u)) + 1u));
                else old[k] = atomicXor(addr, (unsigned long long)(r ? r : 1ull));
            }
            if (a.fetched) {
#pragma unroll
                for (int k = 0; k < U; k++)
                    if (act[k]) __stcs((unsigned long long *)a.fetched + base + (uint64_t)k * blockDim.x, old[k]);
            }
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t *sv = s_val + warp * 32, *so = s_old + warp * 32;
    for (uint64_t base = lo + (uint64_t)warp * 32; base < hi; base += (uint64_t)nwarps * 32) {
        const uint64_t i = base + lane;
        bool active = i < hi;
        uint32_t op = active ? __ldcs(a.ops + i) : 0u;
        const uint64_t w = op & ((1u << 27) - 1u);
        if (active && (w >= a.nwords || ((op >> 27) & 3u) == 3u)) {
            // word outside the table or unknown op code: record it, skip the op
            int *stw = (int *)(a.state + SHMEMG_STATUS_OFF);
            if (atomicCAS(stw, 0, SHMEMG_ERR_INVALID_ARG) == 0) *(volatile int64_t *)(a.state + SHMEMG_STATUS_OFF + 8) = (int64_t)i;
            active = false;
        }
        const uint32_t code = (op >> 27) & 3u;
        const uint64_t r = cb64(a.op_seed, i);
        uint64_t pe, idx;
        if (a.wpp_log2 >= 0) {
            pe = w >> a.wpp_log2;
            idx = w & (a.wpp - 1);
        } else {
            pe = w / a.wpp;
            idx = w - pe * a.wpp;
        }
        unsigned long long *addr = (unsigned long long *)(a.heap + pe * a.H + a.table_off + idx * 8);
        uint64_t old = 0;
        const bool combinable = active && code != 1u;
        const uint32_t agg = (a.flags & SHMEMG_AMO_AGGREGATE) ? __ballot_sync(0xffffffffu, combinable) : 0u;
        if (active && code == 1u) {
            old = atomicCAS(addr, (unsigned long long)cb64(a.table_seed, w), (unsigned long long)r);
        } else if (combinable) {
            const uint64_t v = code == 0u ? (r & ((1u << 20) - 1u)) + 1u : (r ? r : 1ull);
            if (agg) {
                // lanes with the same target and op form one group; the group's ops are
                // applied as one atomic of their combined operand, i.e. consecutively in
                // lane order, and each lane fetches old + (ops of lower lanes)
                const uint64_t key = (uint64_t)addr ^ ((uint64_t)code << 62);
                const uint32_t grp = __match_any_sync(agg, key);
                sv[lane] = v;
                __syncwarp(agg);
                uint64_t pre = 0;
                for (uint32_t m = grp & lt; m; m &= m - 1) {
                    const int j = __ffs(m) - 1;
                    pre = code == 0u ? pre + sv[j] : pre ^ sv[j];
                }
                const int leader = __ffs(grp) - 1;
                if (lane == leader) {
                    uint64_t tot = 0;
                    for (uint32_t m = grp; m; m &= m - 1) {
                        const int j = __ffs(m) - 1;
                        tot = code == 0u ? tot + sv[j] : tot ^ sv[j];
                    }
                    so[lane] = code == 0u ? atomicAdd(addr, (unsigned long long)tot)
                                          : atomicXor(addr, (unsigned long long)tot);
                }
                __syncwarp(agg);
                const uint64_t base_old = so[leader];
                old = code == 0u ? base_old + pre : base_old ^ pre;
                __syncwarp(agg);
            } else {
                old = code == 0u ? atomicAdd(addr, (unsigned long long)v) : atomicXor(addr, (unsigned long long)v);
            }
        }
        if (active && a.fetched) __stcs((unsigned long long *)a.fetched + i, (unsigned long long)old);
    }
}

// Ping-pong between PEs 2k and 2k+1 (one CTA each): put the payload into the peer's
// buf + payload, release-add 1 to the peer's signal, acquire-wait for the own signal.
// (at most 64 registers: 1024 ping-pong CTAs must be co-resident)
__global__ void __launch_bounds__(PP_THREADS, 8) k_pingpong(shmemg_device_ctx_t c, uint64_t buf_off, uint64_t sig_off,
                                                         uint64_t payload, int iters, uint64_t *lat) {
    __shared__ int s_stop;
    const int me = blockIdx.x, peer = me ^ 1, pair = me >> 1;
    const bool pinger = (me & 1) == 0;
    const uint64_t *my_sig = (const uint64_t *)shmemg_d_addr(c, me, sig_off);
    uint64_t *peer_sig = (uint64_t *)shmemg_d_addr(c, peer, sig_off);
    const shmemg_group g = shmemg_d_group_block();
    uint64_t t_start = 0;
    if (threadIdx.x == 0) s_stop = 0;
    __syncthreads();
    for (int t = 0; t < iters; t++) {
        if (pinger) {
            if (threadIdx.x == 0) t_start = shmemg_d_globaltimer();
            shmemg_d_copy_group(g, shmemg_d_addr(c, peer, buf_off + payload), shmemg_d_addr(c, me, buf_off), payload);
            __syncthreads();
            if (threadIdx.x == 0) {
                shmemg_d_fence_gpu();
                shmemg_d_red_release_add_u64(peer_sig, 1);
                if (shmemg_d_signal_wait_until(c, my_sig, SHMEMG_CMP_GE, (uint64_t)t + 1, pair) != SHMEMG_SUCCESS)
                    s_stop = 1;
                if (lat) lat[(uint64_t)pair * iters + t] = shmemg_d_globaltimer() - t_start;
            }
            __syncthreads();
        } else {
            if (threadIdx.x == 0 &&
                shmemg_d_signal_wait_until(c, my_sig, SHMEMG_CMP_GE, (uint64_t)t + 1, pair) != SHMEMG_SUCCESS)
                s_stop = 1;
            __syncthreads();
            if (s_stop) break;
            shmemg_d_copy_group(g, shmemg_d_addr(c, peer, buf_off + payload), shmemg_d_addr(c, me, buf_off), payload);
            __syncthreads();
            if (threadIdx.x == 0) {
                shmemg_d_fence_gpu();
                shmemg_d_red_release_add_u64(peer_sig, 1);
            }
        }
        if (s_stop) break;
    }
}

// The same ping-pong between the two CTAs of a pair inside one cluster, through
// distributed shared memory: the payload is stored straight into the peer's
// shared-memory window and the signal is a word of that window, raised with a
// cluster-scope release add; each side acquire-polls its own window.  At the end each
// PE writes the last payload it received to buf + payload and adds the rounds it
// received to its heap signal word: the heap ends as after the same put_signals into
// the heap.
__global__ void __launch_bounds__(PP_THREADS, 8) k_pingpong_cluster(shmemg_device_ctx_t c, uint64_t buf_off,
                                                                 uint64_t sig_off, uint64_t payload, int iters,
                                                                 uint64_t *lat) {
    extern __shared__ __align__(16) uint8_t s_win[];  // payload bytes, then the signal word
    __shared__ int s_stop;
    const int me = blockIdx.x, pair = me >> 1;
    if (shmemg_d_cluster_nctarank() < 2) {  // launched without clusters: no peer to map
        if (threadIdx.x == 0 && me == 0) shmemg_d_set_status(c, SHMEMG_ERR_UNSUPPORTED, -1);
        return;
    }
    const uint32_t peer_rank = shmemg_d_cluster_ctarank() ^ 1u;
    const bool pinger = (me & 1) == 0;
    uint64_t *my_sig = (uint64_t *)(s_win + ((payload + 15) & ~15ull));
    if (threadIdx.x == 0) {
        *my_sig = 0;
        s_stop = 0;
    }
    shmemg_d_cluster_sync();  // both CTAs started, windows initialised
    const uint8_t *src = shmemg_d_addr(c, me, buf_off);
    uint64_t t_start = 0;
    for (int t = 0; t < iters; t++) {
        if (pinger) {
            if (threadIdx.x == 0) t_start = shmemg_d_globaltimer();
            shmemg_d_putmem_signal_cluster_block(s_win, src, payload, my_sig, 1, SHMEMG_SIGNAL_ADD, peer_rank);
            if (threadIdx.x == 0) {
                if (shmemg_d_signal_wait_until_cluster(c, my_sig, SHMEMG_CMP_GE, (uint64_t)t + 1, pair) != SHMEMG_SUCCESS)
                    s_stop = 1;
                if (lat) lat[(uint64_t)pair * iters + t] = shmemg_d_globaltimer() - t_start;
            }
            __syncthreads();
        } else {
            if (threadIdx.x == 0 &&
                shmemg_d_signal_wait_until_cluster(c, my_sig, SHMEMG_CMP_GE, (uint64_t)t + 1, pair) != SHMEMG_SUCCESS)
                s_stop = 1;
            __syncthreads();
            if (s_stop) break;
            shmemg_d_putmem_signal_cluster_block(s_win, src, payload, my_sig, 1, SHMEMG_SIGNAL_ADD, peer_rank);
        }
        if (s_stop) break;
    }
    // the peer's last update of this window precedes the last signal this CTA acquired;
    // the cluster barrier also keeps both windows alive until both are done
    shmemg_d_cluster_sync();
    if (*my_sig == 0) return;  // nothing received: the heap keeps its contents
    // (the window is shared memory: read it with shared-space loads, never ld.global)
    shmemg_d_copy_from_cluster(shmemg_d_group_block(), shmemg_d_addr(c, me, buf_off + payload), s_win,
                               shmemg_d_cluster_ctarank(), payload);
    if (threadIdx.x == 0) {
        uint64_t *hs = (uint64_t *)shmemg_d_addr(c, me, sig_off);
        *hs += *my_sig;
    }
}

__global__ void k_time(uint64_t *out) { *out = shmemg_d_globaltimer(); }

}  // namespace shmemg

using namespace shmemg;

extern "C" {

int shmemg_amo_stream(int64_t *table, uint64_t words_per_pe, const uint32_t *ops, uint64_t nops, uint64_t op_seed,
                      uint64_t table_seed, int64_t *fetched, uint32_t flags, void *stream) {
    if (int rc = check_init()) return rc;
    State &S = st();
    if (words_per_pe == 0 || (nops && !ops)) return SHMEMG_ERR_INVALID_ARG;
    if ((uint64_t)S.npes * words_per_pe > (1ull << 27)) return SHMEMG_ERR_INVALID_ARG;  // 27-bit word index
    uint64_t off;
    if (sym_offset(table, words_per_pe * 8, &off) || (off & 7)) return SHMEMG_ERR_NOT_SYMMETRIC;
    if (flags & ~SHMEMG_AMO_AGGREGATE) return SHMEMG_ERR_INVALID_ARG;
    if (nops == 0) return SHMEMG_SUCCESS;
    AmoArgs a;
    a.heap = S.heap;
    a.H = S.H;
    a.table_off = off;
    a.wpp = words_per_pe;
    a.wpp_log2 = (words_per_pe & (words_per_pe - 1)) ? -1 : __builtin_ctzll(words_per_pe);
    a.npes = S.npes;
    a.ops = ops;
    a.nops = nops;
    a.op_seed = op_seed;
    a.table_seed = table_seed;
    a.fetched = fetched;
    a.flags = flags;
    a.nwords = (uint64_t)S.npes * words_per_pe;
    a.state = S.base;
    k_amo_stream<<<S.npes, AMO_THREADS, 0, to_stream(stream)>>>(a);
    return cuda_rc(cudaGetLastError());
}


int shmemg_pingpong(void *buf, uint64_t *sig, uint64_t payload, int npairs, int iters, uint64_t *lat_ns, void *stream) {
    if (int rc = check_init()) return rc;
    State &S = st();
    if (npairs < 1 || iters < 0 || 2 * npairs > S.npes) return SHMEMG_ERR_INVALID_ARG;
    if (S.pe_mode != SHMEMG_PE_MODE_CTA) return SHMEMG_ERR_UNSUPPORTED;
    uint64_t boff, soff;
    if (sym_offset(buf, 2 * payload, &boff) || sym_offset(sig, 8, &soff) || (soff & 7)) return SHMEMG_ERR_NOT_SYMMETRIC;
    shmemg_device_ctx_t c = device_ctx();
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pingpong, PP_THREADS, 0);
    if ((int64_t)per_sm * S.sm_count < 2 * npairs) return SHMEMG_ERR_UNSUPPORTED;
    void *args[] = {(void *)&c, (void *)&boff, (void *)&soff, (void *)&payload, (void *)&iters, (void *)&lat_ns};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * npairs);
    cfg.blockDim = dim3(PP_THREADS);
    cfg.stream = to_stream(stream);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cuda_rc(cudaLaunchKernelExC(&cfg, (const void *)k_pingpong, args));
}

int shmemg_pingpong_cluster(void *buf, uint64_t *sig, uint64_t payload, int npairs, int iters, uint64_t *lat_ns,
                            void *stream) {
    if (int rc = check_init()) return rc;
    State &S = st();
    if (npairs < 1 || iters < 0 || 2 * npairs > S.npes || payload > SHMEMG_PINGPONG_CLUSTER_MAX) return SHMEMG_ERR_INVALID_ARG;
    if (S.pe_mode != SHMEMG_PE_MODE_CTA || S.cluster_dim < 2 || (2 * npairs) % S.cluster_dim) return SHMEMG_ERR_UNSUPPORTED;
    uint64_t boff, soff;
    if (sym_offset(buf, 2 * payload, &boff) || sym_offset(sig, 8, &soff) || (soff & 7)) return SHMEMG_ERR_NOT_SYMMETRIC;
    shmemg_device_ctx_t c = device_ctx();
    const size_t smem = ((payload + 15) & ~15ull) + 16;
    if (smem > 48 * 1024 && cudaFuncSetAttribute((const void *)k_pingpong_cluster,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return SHMEMG_ERR_UNSUPPORTED;
    }
    void *args[] = {(void *)&c, (void *)&boff, (void *)&soff, (void *)&payload, (void *)&iters, (void *)&lat_ns};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * npairs);
    cfg.blockDim = dim3(PP_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = to_stream(stream);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S.cluster_dim;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // no cooperative launch needed: the two CTAs of a pair are in one cluster, which the
    // hardware always schedules at once, and pairs never wait on each other
    return cuda_rc(cudaLaunchKernelExC(&cfg, (const void *)k_pingpong_cluster, args));
}

int shmemg_device_time_ns(uint64_t *out) {
    if (!out) return SHMEMG_ERR_INVALID_ARG;
    uint64_t *d = nullptr;
    int rc = cuda_rc(cudaMallocHost(&d, 8));
    if (rc) return rc;
    k_time<<<1, 1>>>(d);
    rc = cuda_rc(cudaDeviceSynchronize());
    if (!rc) *out = *d;
    cudaFreeHost(d);
    return rc;
}

}  // extern "C"
