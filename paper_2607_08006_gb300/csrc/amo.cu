// Device-initiated AMO stress stream and put-with-signal ping-pong (paper Sec. 2.1
// atomics; Sec. 6.3 "atomicity does not imply ordering"; Sec. 7 put-signal; case
// study 2 of Sec. 4.4: fine-grained atomics and polling flags in graph analytics).
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace shmemg {

constexpr int AMO_THREADS = 256;
constexpr int PP_THREADS = 128;

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

// Block-combined stream.  PE p's range [p*nops/npes, (p+1)*nops/npes) is cut into tiles
// of CB_TILE consecutive ops; a persistent grid (as many CTAs as are resident at once)
// walks the tiles of all PEs, a CTA acting as the tile's PE (op j of a tile at thread
// j % blockDim.x, CB_U per thread).  Ops of one tile with the same target word and
// op code form a group through an open-addressing table in shared memory; the group is
// applied to the word by ONE global atomic, and its ops take consecutive places in the
// serial order (the order of their shared-memory atomics):
//   fetch_add / fetch_xor -- each op's shared atomic on the group's accumulator returns
//     the combined operand of the ops before it (its prefix); the op that inserted the
//     key applies the total and every op fetches old + prefix (old ^ prefix);
//   compare_swap -- all ops on word w compare against the same initial value c, so after
//     the first op of a group the word holds either its old value (old != c) or the first
//     op's swap value r0; provided no swap value equals c, the later ops all fail and
//     fetch that value.  The first op (shared counter 0) issues CAS(c, r0); an op whose
//     swap value equals c is applied on its own.
// With Zipf-distributed targets this turns the serialised atomics on the hottest words
// (about 11% of all ops land on one word at s = 1.1 over 2^27 words) into one atomic per
// tile and group.
constexpr int CB_THREADS = 256;
constexpr int CB_U = 4;
constexpr int CB_TILE = CB_THREADS * CB_U;
constexpr int CB_SLOTS_LOG2 = CB_TILE == 1024 ? 11 : CB_TILE == 2048 ? 12 : CB_TILE == 512 ? 10 : 13;
constexpr int CB_SLOTS = 1 << CB_SLOTS_LOG2;   // load factor <= 1/2
static_assert(CB_SLOTS >= 2 * CB_TILE, "table load factor");
constexpr int CB_MIN_BLOCKS = 4;
constexpr size_t CB_SMEM = (size_t)CB_SLOTS * (8 + 4);

__device__ __forceinline__ unsigned long long *amo_addr(const AmoArgs &a, uint32_t w) {
    const uint64_t pe = a.wpp_log2 >= 0 ? (uint64_t)w >> a.wpp_log2 : w / a.wpp;
    return (unsigned long long *)(a.heap + pe * a.H + a.table_off + (w - pe * a.wpp) * 8);
}

__global__ void __launch_bounds__(CB_THREADS, CB_MIN_BLOCKS) k_amo_combine(AmoArgs a) {
    extern __shared__ __align__(16) unsigned char cb_smem[];
    unsigned long long *s_acc = (unsigned long long *)cb_smem;   // accumulator / counter, then the fetched base
    uint32_t *s_key = (uint32_t *)(s_acc + CB_SLOTS);            // (word << 2 | code) + 1, 0 = empty
    __shared__ uint64_t s_tile[2];                    // [base, hi) of the CTA's current tile
    const uint64_t tiles_per_pe = (a.nops / (uint64_t)a.npes + 1 + CB_TILE - 1) / CB_TILE;
    const uint64_t ntiles = tiles_per_pe * (uint64_t)a.npes;
    auto tile = [&](uint64_t t) {   // thread 0: tile t covers ops [base, hi) of its PE's range
        const uint64_t p = t / tiles_per_pe;
        s_tile[0] = a.nops * p / (uint64_t)a.npes + (t - p * tiles_per_pe) * CB_TILE;
        s_tile[1] = a.nops * (p + 1) / (uint64_t)a.npes;
    };
    for (int j = threadIdx.x; j < CB_SLOTS; j += blockDim.x) {
        s_key[j] = 0u;
        s_acc[j] = 0ull;
    }
    if (threadIdx.x == 0 && blockIdx.x < ntiles) tile(blockIdx.x);
    __syncthreads();
    // per op: word, then slot (bits 0..CB_SLOTS_LOG2-1), role (next 2 bits: 0 inactive,
    // 1 group member, 2 group issuer, 3 applied on its own) and code (2 bits); the prefix
    constexpr int ROLE = CB_SLOTS_LOG2, CODE = CB_SLOTS_LOG2 + 2;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t base = s_tile[0], hi = s_tile[1];
        if (base >= hi) {            // uniform across the CTA
            __syncthreads();
            if (threadIdx.x == 0 && t + gridDim.x < ntiles) tile(t + gridDim.x);
            __syncthreads();
            continue;
        }
        uint32_t w[CB_U], sr[CB_U];
        unsigned long long pre[CB_U];
#pragma unroll
        for (int k = 0; k < CB_U; k++) {
            const uint64_t i = base + (uint64_t)k * blockDim.x + threadIdx.x;
            sr[k] = 0u;
            w[k] = 0u;
            pre[k] = 0ull;
            if (i >= hi) continue;
            const uint32_t op = __ldcs(a.ops + i);
            w[k] = op & ((1u << 27) - 1u);
            const uint32_t code = (op >> 27) & 3u;
            if (w[k] >= a.nwords || code == 3u) {
                int *stw = (int *)(a.state + SHMEMG_STATUS_OFF);
                if (atomicCAS(stw, 0, SHMEMG_ERR_INVALID_ARG) == 0) *(volatile int64_t *)(a.state + SHMEMG_STATUS_OFF + 8) = (int64_t)i;
                continue;
            }
            const uint64_t r = cb64(a.op_seed, i);
            unsigned long long opnd;
            if (code == 1u) {
                const uint64_t c = cb64(a.table_seed, w[k]);
                if (r == c) {
                    sr[k] = 3u << ROLE | code << CODE;
                    const unsigned long long old = atomicCAS(amo_addr(a, w[k]), c, r);
                    if (a.fetched) __stcs((unsigned long long *)a.fetched + i, old);
                    continue;
                }
                opnd = 1ull;
            } else {
                opnd = code == 0u ? (r & ((1u << 20) - 1u)) + 1u : (r ? r : 1ull);
            }
            const uint32_t key = (w[k] << 2 | code) + 1u;
            uint32_t h = (key * 0x9E3779B1u) >> (32 - CB_SLOTS_LOG2);
            uint32_t prev = 0;
            for (int q = 0; q < CB_SLOTS; q++) {   // an empty or matching slot always exists
                prev = atomicCAS(&s_key[h], 0u, key);
                if (prev == 0u || prev == key) break;
                h = (h + 1) & (CB_SLOTS - 1);
            }
            pre[k] = code == 2u ? atomicXor(&s_acc[h], opnd) : atomicAdd(&s_acc[h], opnd);
            const uint32_t role = (code == 1u ? pre[k] == 0ull : prev == 0u) ? 2u : 1u;
            sr[k] = h | role << ROLE | code << CODE;
        }
        __syncthreads();
        // issuers apply their group (all atomics issued before any result is used)
        unsigned long long old[CB_U];
#pragma unroll
        for (int k = 0; k < CB_U; k++) {
            old[k] = 0ull;
            if ((sr[k] >> ROLE & 3u) != 2u) continue;
            const uint32_t code = sr[k] >> CODE & 3u;
            unsigned long long *p = amo_addr(a, w[k]);
            if (code == 1u) {
                old[k] = atomicCAS(p, cb64(a.table_seed, w[k]), cb64(a.op_seed, base + (uint64_t)k * blockDim.x + threadIdx.x));
            } else {
                const unsigned long long tot = s_acc[sr[k] & (CB_SLOTS - 1)];
                old[k] = code == 0u ? atomicAdd(p, tot) : atomicXor(p, tot);
            }
        }
#pragma unroll
        for (int k = 0; k < CB_U; k++) {
            if ((sr[k] >> ROLE & 3u) != 2u) continue;
            const uint32_t code = sr[k] >> CODE & 3u;
            unsigned long long b = old[k];
            if (code == 1u) {   // what the later ops of the group fetch
                const uint64_t c = cb64(a.table_seed, w[k]);
                b = old[k] == c ? cb64(a.op_seed, base + (uint64_t)k * blockDim.x + threadIdx.x) : old[k];
            }
            s_acc[sr[k] & (CB_SLOTS - 1)] = b;
            if (a.fetched)
                __stcs((unsigned long long *)a.fetched + base + (uint64_t)k * blockDim.x + threadIdx.x,
                       code == 0u ? old[k] + pre[k] : code == 2u ? (old[k] ^ pre[k]) : old[k]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < CB_U; k++) {
            if ((sr[k] >> ROLE & 3u) != 1u || !a.fetched) continue;
            const uint32_t code = sr[k] >> CODE & 3u;
            const unsigned long long b = s_acc[sr[k] & (CB_SLOTS - 1)];
            __stcs((unsigned long long *)a.fetched + base + (uint64_t)k * blockDim.x + threadIdx.x,
                   code == 0u ? b + pre[k] : code == 2u ? (b ^ pre[k]) : b);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < CB_U; k++)
            if ((sr[k] >> ROLE & 3u) == 2u) {
                s_key[sr[k] & (CB_SLOTS - 1)] = 0u;
                s_acc[sr[k] & (CB_SLOTS - 1)] = 0ull;
            }
        if (threadIdx.x == 0 && t + gridDim.x < ntiles) tile(t + gridDim.x);
        __syncthreads();
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
    if (flags & ~(SHMEMG_AMO_AGGREGATE | SHMEMG_AMO_COMBINE_BLOCK)) return SHMEMG_ERR_INVALID_ARG;
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
    if (flags & SHMEMG_AMO_COMBINE_BLOCK) {
        static int per_sm = 0;
        if (!per_sm) {
            if (cudaFuncSetAttribute((const void *)k_amo_combine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CB_SMEM) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_amo_combine, CB_THREADS, CB_SMEM) != cudaSuccess || per_sm < 1)
                per_sm = 1;
        }
        const uint64_t tiles = ((nops / S.npes + 1 + CB_TILE - 1) / CB_TILE) * S.npes;
        const int grid = (int)std::min<uint64_t>(tiles, (uint64_t)per_sm * S.sm_count);
        k_amo_combine<<<grid, CB_THREADS, CB_SMEM, to_stream(stream)>>>(a);
    } else k_amo_stream<<<S.npes, AMO_THREADS, 0, to_stream(stream)>>>(a);
    return cuda_rc(cudaGetLastError());
}


int shmemg_pingpong(void *buf, uint64_t *sig, uint64_t payload, int npairs, int iters, uint64_t *lat_ns, void *stream) {
    if (int rc = check_init()) return rc;
    State &S = st();
    if (npairs < 1 || iters < 0 || 2 * (int64_t)npairs > S.npes) return SHMEMG_ERR_INVALID_ARG;
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
    if (npairs < 1 || iters < 0 || 2 * (int64_t)npairs > S.npes || payload > SHMEMG_PINGPONG_CLUSTER_MAX) return SHMEMG_ERR_INVALID_ARG;
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
