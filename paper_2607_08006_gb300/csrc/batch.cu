// Batched uneven collectives: many teams' sum all-reduces in one persistent launch
// captured in a CUDA graph (a batching extension of the team reductions the paper
// inherits from OpenSHMEM 1.6, Sec. 6.3).
//
// Work items are (team, tile) pairs planned on the host, largest team first (cost =
// members x elements x bytes); CTAs of a persistent grid take items from a device
// counter.  Each item is a slice-owner reduction of one tile over the team's members:
// fp32 by the fixed rank-pairwise tree, int64 exactly, bf16/e4m3 payloads dequantised
// and accumulated with Neumaier's compensated sum.  The last CTA to leave resets the
// counters, so graph replays need no memset node.  The autotuner times candidate
// (tile, CTAs per SM) plans with CUDA events and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "quant_dev.cuh"

namespace shmemg {

constexpr int B_THREADS = 256;
constexpr int B_DEEP_QM = 16;
// Two kernels (the plan's `deep` picks one): the lean one holds 85 registers for 3 CTAs per
// SM, with 16 members' loads in flight in the fp32 tree and 8 quantised members loaded
// ahead; the deep one holds 128 registers for 2 CTAs per SM and loads further ahead.
template <int MINB> struct BShape;
template <> struct BShape<3> { static constexpr int TREE_MAXB = 4, QM = 8; };
template <> struct BShape<2> { static constexpr int TREE_MAXB = 4, QM = B_DEEP_QM; };
enum BKind { BK_F32 = 0, BK_I64 = 1, BK_BF16 = 2, BK_E4M3 = 3 };

struct BTeam {
    int32_t start, size, kind, vec;
    uint64_t n, d_off, s_off, sc_off;
};

struct BArgs {
    uint8_t *heap;
    uint64_t H;
    const BTeam *teams;
    const uint2 *items;   // (team, tile)
    uint32_t nitems;
    uint32_t tile;        // elements per item
    uint32_t *counter;    // [0] next item, [1] CTAs done
};

// quantised tile: full chunks of blockDim x E elements accumulate into shared memory (two
// buffers, alternated across the CTA's chunks) and are bulk-stored to every member (bit 1
// of t.vec: 16-byte aligned codes and outputs); the rest runs E (or 4) elements per thread
template <int FMT, int M>
__device__ __forceinline__ void batch_qsum(const BArgs &a, const BTeam &t, uint64_t e0, uint64_t e1, float (*s_out)[B_THREADS * 16],
                                           int &buf) {
    constexpr int E = QWide<FMT>::E;
    const uint64_t CH = (uint64_t)blockDim.x * E;
    uint64_t f0 = e0;
    if (t.vec & 2) {
        for (; f0 + CH <= e1; f0 += CH) {
            qsum_chunk_tma<FMT, M>(a.heap, a.H, t.start, 1, t.size, t.d_off, t.s_off, t.sc_off, f0, s_out[buf]);
            buf ^= 1;
        }
    }
    for (uint64_t q = f0 / E + threadIdx.x; q * E < e1; q += blockDim.x) {
        const uint64_t f = q * E;
        if ((t.vec & 2) && f + E <= e1) {
            qsum_wide<FMT, M>(a.heap, a.H, t.start, 1, t.size, t.d_off, t.s_off, t.sc_off, f);
        } else {
            for (int k = 0; k < E / 4 && f + 4 * k < e1; k++)
                qsum4<FMT>(a.heap, a.H, t.start, 1, t.size, t.d_off, t.s_off, t.sc_off, f + 4 * k, t.n,
                           (t.vec & 1) && f + 4 * k + 4 <= t.n);
        }
    }
}

template <int MINB>
__device__ __forceinline__ void batch_item(const BArgs &a, const BTeam &t, uint64_t e0, uint64_t e1, float (*s_out)[B_THREADS * 16],
                                           int &buf) {
    const shmemg_group g = {threadIdx.x, blockDim.x};
    if (t.kind == BK_F32) {
        shmemg_d_reduce_elems_t<float, float4, BShape<MINB>::TREE_MAXB>(g, a.heap, a.H, t.start, 1, t.size, t.d_off, t.s_off, e0, e1,
                                                         SHMEMG_SUM);
    } else if (t.kind == BK_I64) {
        shmemg_d_reduce_elems_t<int64_t, longlong2>(g, a.heap, a.H, t.start, 1, t.size, t.d_off, t.s_off, e0, e1,
                                                    SHMEMG_SUM);
    } else {
        if (t.kind == BK_E4M3) batch_qsum<SHMEMG_FMT_E4M3, BShape<MINB>::QM>(a, t, e0, e1, s_out, buf);
        else batch_qsum<SHMEMG_FMT_BF16, BShape<MINB>::QM>(a, t, e0, e1, s_out, buf);
    }
}

template <int MINB>
__global__ void __launch_bounds__(B_THREADS, MINB) k_batch(BArgs a) {
    __shared__ uint32_t s_item;
    __shared__ __align__(128) float s_out[2][B_THREADS * 16];  // two quantised chunks (E <= 16), alternated
    int buf = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&a.counter[0], 1u);
        __syncthreads();
        const uint32_t it = s_item;
        __syncthreads();
        if (it >= a.nitems) break;
        const uint2 item = a.items[it];
        const BTeam t = a.teams[item.x];
        const uint64_t e0 = (uint64_t)item.y * a.tile;
        const uint64_t e1 = e0 + a.tile < t.n ? e0 + a.tile : t.n;
        batch_item<MINB>(a, t, e0, e1, s_out, buf);
    }
    if (threadIdx.x == 0) {
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // this CTA's bulk stores are done
        // every CTA has drawn its final (out-of-range) item before it counts itself
        // done, so the last one can reset both words for the next launch
        __threadfence();
        if (atomicAdd(&a.counter[1], 1u) == gridDim.x - 1) {
            a.counter[0] = 0;
            a.counter[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace shmemg

using namespace shmemg;

struct shmemg_batch_s {
    std::vector<BTeam> teams;
    std::vector<uint64_t> cost;
    BTeam *d_teams = nullptr;
    uint2 *d_items = nullptr;
    uint32_t *d_counter = nullptr;
    uint32_t nitems = 0;
    shmemg_tune_t tune{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid = 0;
};

static void free_graph(shmemg_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// (re)plan items for the batch's tile size, upload them and capture the graph
static int plan_and_capture(shmemg_batch_s *b) {
    State &S = st();
    const uint32_t tile = (uint32_t)b->tune.tile_elems;
    std::vector<int> order(b->teams.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
    std::vector<uint2> items;
    for (int t : order) {
        uint64_t tiles = (b->teams[t].n + tile - 1) / tile;
        for (uint64_t k = 0; k < tiles; k++) items.push_back(make_uint2((unsigned)t, (unsigned)k));
    }
    if (items.size() >= (1ull << 31)) return SHMEMG_ERR_INVALID_ARG;
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    int rc = cuda_rc(cudaMalloc(&b->d_items, sizeof(uint2) * (items.size() ? items.size() : 1)));
    if (rc) return rc;
    if ((rc = cuda_rc(cudaMemcpy(b->d_items, items.data(), sizeof(uint2) * items.size(), cudaMemcpyHostToDevice))))
        return rc;
    b->nitems = (uint32_t)items.size();
    int per_sm = 0;
    const void *kfn = b->tune.deep ? (const void *)k_batch<2> : (const void *)k_batch<3>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, B_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    int want = b->tune.ctas_per_sm > 0 ? std::min(b->tune.ctas_per_sm, per_sm) : per_sm;
    b->grid = want * S.sm_count;
    if ((uint32_t)b->grid > b->nitems) b->grid = (int)std::max<uint32_t>(b->nitems, 1u);
    free_graph(b);
    cudaStream_t cs;
    if ((rc = cuda_rc(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)))) return rc;
    BArgs a;
    a.heap = S.heap;
    a.H = S.H;
    a.teams = b->d_teams;
    a.items = b->d_items;
    a.nitems = b->nitems;
    a.tile = tile;
    a.counter = b->d_counter;
    rc = cuda_rc(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    if (!rc) {
        if (b->tune.deep) k_batch<2><<<b->grid, B_THREADS, 0, cs>>>(a);
        else k_batch<3><<<b->grid, B_THREADS, 0, cs>>>(a);
        cudaError_t le = cudaGetLastError();
        cudaError_t ee = cudaStreamEndCapture(cs, &b->graph);
        rc = cuda_rc(le != cudaSuccess ? le : ee);
    }
    if (!rc) rc = cuda_rc(cudaGraphInstantiate(&b->exec, b->graph, 0));
    cudaStreamDestroy(cs);
    return rc;
}

extern "C" {

int shmemg_batch_create(const shmemg_coll_desc_t *descs, int count, const shmemg_tune_t *tune, shmemg_batch_t *out) {
    if (int rc = check_init()) return rc;
    if (!out || count < 1 || !descs) return SHMEMG_ERR_INVALID_ARG;
    State &S = st();
    auto *b = new shmemg_batch_s();
    for (int i = 0; i < count; i++) {
        const shmemg_coll_desc_t &d = descs[i];
        BTeam t;
        memset(&t, 0, sizeof(t));
        if (d.size < 1 || d.start < 0 || (int64_t)d.start + d.size > S.npes || d.n == 0) { delete b; return SHMEMG_ERR_INVALID_ARG; }
        t.start = d.start;
        t.size = d.size;
        t.n = d.n;
        uint64_t in_es, out_es = 4;
        if (d.dtype == SHMEMG_INT64) { t.kind = BK_I64; in_es = 8; out_es = 8; }
        else if (d.dtype == SHMEMG_FLOAT && d.fmt < 0) { t.kind = BK_F32; in_es = 4; }
        else if (d.dtype == SHMEMG_FLOAT && d.fmt == SHMEMG_FMT_BF16) { t.kind = BK_BF16; in_es = 2; }
        else if (d.dtype == SHMEMG_FLOAT && d.fmt == SHMEMG_FMT_E4M3) { t.kind = BK_E4M3; in_es = 1; }
        else { delete b; return SHMEMG_ERR_INVALID_ARG; }
        if (sym_offset(d.dst, d.n * out_es, &t.d_off) || sym_offset(d.src, d.n * in_es, &t.s_off)) {
            delete b;
            return SHMEMG_ERR_NOT_SYMMETRIC;
        }
        if ((t.d_off % out_es) || (t.s_off % in_es)) { delete b; return SHMEMG_ERR_INVALID_ARG; }
        if (t.kind >= BK_BF16) {
            if (!d.scales || sym_offset(d.scales, (d.n + 127) / 128 * 4, &t.sc_off) || (t.sc_off & 3)) {
                delete b;
                return SHMEMG_ERR_NOT_SYMMETRIC;
            }
            t.vec = ((t.d_off & 15) == 0 && (t.s_off & (t.kind == BK_E4M3 ? 3 : 7)) == 0 ? 1 : 0) |
                    ((t.d_off & 15) == 0 && (t.s_off & 15) == 0 ? 2 : 0);
        }
        b->teams.push_back(t);
        b->cost.push_back((uint64_t)d.size * d.n * (in_es + out_es));
    }
    b->tune.tile_elems = tune && tune->tile_elems > 0 ? tune->tile_elems : 16384;
    b->tune.ctas_per_sm = tune ? tune->ctas_per_sm : 0;
    b->tune.threads = B_THREADS;
    b->tune.deep = tune && tune->deep ? 1 : 0;
    if (b->tune.tile_elems % 128) { delete b; return SHMEMG_ERR_INVALID_ARG; }
    int rc = cuda_rc(cudaMalloc(&b->d_teams, sizeof(BTeam) * b->teams.size()));
    if (!rc) rc = cuda_rc(cudaMemcpy(b->d_teams, b->teams.data(), sizeof(BTeam) * b->teams.size(), cudaMemcpyHostToDevice));
    if (!rc) rc = cuda_rc(cudaMalloc(&b->d_counter, 2 * sizeof(uint32_t)));
    if (!rc) rc = cuda_rc(cudaMemset(b->d_counter, 0, 2 * sizeof(uint32_t)));
    if (!rc) rc = plan_and_capture(b);
    if (rc) {
        shmemg_batch_destroy(b);
        return rc;
    }
    *out = b;
    return SHMEMG_SUCCESS;
}

int shmemg_batch_launch(shmemg_batch_t b, void *stream) {
    if (int rc = check_init()) return rc;
    if (!b || !b->exec) return SHMEMG_ERR_INVALID_ARG;
    return cuda_rc(cudaGraphLaunch(b->exec, to_stream(stream)));
}

int shmemg_batch_autotune(shmemg_batch_t b, void *stream, shmemg_tune_t *chosen) {
    if (int rc = check_init()) return rc;
    if (!b) return SHMEMG_ERR_INVALID_ARG;
    cudaStream_t s = to_stream(stream);
    const int tiles[] = {2048, 4096, 8192, 32768, 131072};
    const int ctas[] = {1, 2, 0, -1};  // (-1: the deep kernel at its 2 CTAs per SM)
    shmemg_tune_t best = b->tune;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = SHMEMG_SUCCESS;
    for (int t : tiles) {
        for (int c : ctas) {
            b->tune.tile_elems = t;
            b->tune.ctas_per_sm = c < 0 ? 0 : c;
            b->tune.deep = c < 0 ? 1 : 0;
            if ((rc = plan_and_capture(b))) break;
            cudaGraphLaunch(b->exec, s);  // warm-up
            cudaEventRecord(e0, s);
            for (int k = 0; k < 3; k++) cudaGraphLaunch(b->exec, s);
            cudaEventRecord(e1, s);
            if ((rc = cuda_rc(cudaEventSynchronize(e1)))) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = b->tune;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->tune = best;
    if ((rc = plan_and_capture(b))) return rc;
    if (chosen) *chosen = best;
    return SHMEMG_SUCCESS;
}

int shmemg_batch_destroy(shmemg_batch_t b) {
    if (!b) return SHMEMG_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    free_graph(b);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_teams) cudaFree(b->d_teams);
    if (b->d_counter) cudaFree(b->d_counter);
    delete b;
    return SHMEMG_SUCCESS;
}

}  // extern "C"

// ================================================================ allocation-free variant
// The batched reduce above keeps its team table, work items and work counters in
// device memory that shmemg_batch_create allocates.  shmemg_batch_reduce_noalloc runs
// the same kernel with those three in one fixed array compiled into the library, so a
// call allocates nothing.  Every GPU that loads the library holds the array until the
// process exits; all calls share it.
namespace shmemg {

struct NoallocScratch {
    BTeam teams[SHMEMG_NOALLOC_MAX_TEAMS];
    uint2 items[SHMEMG_NOALLOC_MAX_ITEMS];
    uint32_t counter[2];
};

static __device__ __align__(256) uint8_t g_noalloc_scratch[sizeof(NoallocScratch)];

// host staging of one call's table and items (no host heap allocation per call)
static BTeam g_noalloc_teams_h[SHMEMG_NOALLOC_MAX_TEAMS];
static uint2 g_noalloc_items_h[SHMEMG_NOALLOC_MAX_ITEMS];
static uint64_t g_noalloc_cost_h[SHMEMG_NOALLOC_MAX_TEAMS];
static int g_noalloc_order_h[SHMEMG_NOALLOC_MAX_TEAMS];
static std::mutex g_noalloc_mu;
constexpr int NOALLOC_MAX_DEVICES = 64;
static NoallocScratch *g_noalloc_dev[NOALLOC_MAX_DEVICES];

// device address of the array on the current device; looked up once per device
static int noalloc_scratch(NoallocScratch **out) {
    int dev = 0;
    int rc = cuda_rc(cudaGetDevice(&dev));
    if (rc) return rc;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SHMEMG_ERR_UNSUPPORTED;
    if (!g_noalloc_dev[dev]) {
        void *p = nullptr;
        if ((rc = cuda_rc(cudaGetSymbolAddress(&p, g_noalloc_scratch)))) return rc;
        g_noalloc_dev[dev] = (NoallocScratch *)p;
    }
    *out = g_noalloc_dev[dev];
    return SHMEMG_SUCCESS;
}

}  // namespace shmemg

extern "C" int shmemg_batch_reduce_noalloc(const shmemg_coll_desc_t *descs, int count, int tile_elems, void *stream) {
    if (int rc = check_init()) return rc;
    if (!descs || count < 1) return SHMEMG_ERR_INVALID_ARG;
    if (count > SHMEMG_NOALLOC_MAX_TEAMS) return SHMEMG_ERR_INVALID_ARG;  // more teams than the array holds
    const uint32_t tile = tile_elems > 0 ? (uint32_t)tile_elems : 16384u;
    if (tile % 128) return SHMEMG_ERR_INVALID_ARG;
    State &S = st();
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocScratch *d = nullptr;
    if (int rc = noalloc_scratch(&d)) return rc;
    uint64_t nitems = 0;
    for (int i = 0; i < count; i++) {
        const shmemg_coll_desc_t &c = descs[i];
        BTeam &t = g_noalloc_teams_h[i];
        memset(&t, 0, sizeof(t));
        if (c.size < 1 || c.start < 0 || (int64_t)c.start + c.size > S.npes || c.n == 0) return SHMEMG_ERR_INVALID_ARG;
        t.start = c.start;
        t.size = c.size;
        t.n = c.n;
        uint64_t in_es, out_es = 4;
        if (c.dtype == SHMEMG_INT64) { t.kind = BK_I64; in_es = 8; out_es = 8; }
        else if (c.dtype == SHMEMG_FLOAT && c.fmt < 0) { t.kind = BK_F32; in_es = 4; }
        else if (c.dtype == SHMEMG_FLOAT && c.fmt == SHMEMG_FMT_BF16) { t.kind = BK_BF16; in_es = 2; }
        else if (c.dtype == SHMEMG_FLOAT && c.fmt == SHMEMG_FMT_E4M3) { t.kind = BK_E4M3; in_es = 1; }
        else return SHMEMG_ERR_INVALID_ARG;
        if (sym_offset(c.dst, c.n * out_es, &t.d_off) || sym_offset(c.src, c.n * in_es, &t.s_off))
            return SHMEMG_ERR_NOT_SYMMETRIC;
        if ((t.d_off % out_es) || (t.s_off % in_es)) return SHMEMG_ERR_INVALID_ARG;
        if (t.kind >= BK_BF16) {
            if (!c.scales || sym_offset(c.scales, (c.n + 127) / 128 * 4, &t.sc_off) || (t.sc_off & 3))
                return SHMEMG_ERR_NOT_SYMMETRIC;
            t.vec = ((t.d_off & 15) == 0 && (t.s_off & (t.kind == BK_E4M3 ? 3 : 7)) == 0 ? 1 : 0) |
                    ((t.d_off & 15) == 0 && (t.s_off & 15) == 0 ? 2 : 0);
        }
        g_noalloc_cost_h[i] = (uint64_t)c.size * c.n * (in_es + out_es);
        g_noalloc_order_h[i] = i;
        nitems += (c.n + tile - 1) / tile;
    }
    if (nitems > SHMEMG_NOALLOC_MAX_ITEMS) return SHMEMG_ERR_INVALID_ARG;  // more work items than the array holds
    std::stable_sort(g_noalloc_order_h, g_noalloc_order_h + count,
                     [](int x, int y) { return g_noalloc_cost_h[x] > g_noalloc_cost_h[y]; });
    uint32_t k = 0;
    for (int j = 0; j < count; j++) {
        const int t = g_noalloc_order_h[j];
        const uint64_t tiles = (g_noalloc_teams_h[t].n + tile - 1) / tile;
        for (uint64_t q = 0; q < tiles; q++) g_noalloc_items_h[k++] = make_uint2((unsigned)t, (unsigned)q);
    }
    cudaStream_t s = to_stream(stream);
    int rc = cuda_rc(cudaMemcpyAsync(d->teams, g_noalloc_teams_h, sizeof(BTeam) * count, cudaMemcpyHostToDevice, s));
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(d->items, g_noalloc_items_h, sizeof(uint2) * k, cudaMemcpyHostToDevice, s));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(d->counter, 0, sizeof(d->counter), s));  // work counters start at zero
    if (rc) return rc;
    BArgs a;
    a.heap = S.heap;
    a.H = S.H;
    a.teams = d->teams;
    a.items = d->items;
    a.nitems = k;
    a.tile = tile;
    a.counter = d->counter;
    int grid = ctas_for((const void *)k_batch<3>, B_THREADS, 0);
    if ((uint32_t)grid > k) grid = (int)k;
    k_batch<3><<<grid, B_THREADS, 0, s>>>(a);
    return cuda_rc(cudaGetLastError());
}
