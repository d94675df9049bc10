// Heap carve-up, symmetric allocation, teams, capability query, status and ordering
// calls of the C ABI (paper Sec. 6.1 memory model, 6.2 contexts/teams, 6.4 ordering,
// 6.5 capability discovery).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "internal.h"

namespace shmemg {

static State g_state;
State &st() { return g_state; }

static thread_local std::string g_cuda_msg;

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return SHMEMG_SUCCESS;
    g_cuda_msg = cudaGetErrorString(e);
    return SHMEMG_ERR_CUDA;
}

shmemg_device_ctx_t device_ctx() {
    shmemg_device_ctx_t c;
    memset(&c, 0, sizeof(c));
    c.heap = g_state.heap;
    c.pe_stride = g_state.H;
    c.npes = g_state.npes;
    c.pe_mode = g_state.pe_mode;
    c.cluster_dim = g_state.cluster_dim;
    c.state = g_state.base;
    c.timeout_ns = g_state.timeout_ns;
    return c;
}

int check_init() { return g_state.init ? SHMEMG_SUCCESS : SHMEMG_ERR_NOT_INITIALIZED; }

int sym_offset(const void *p, uint64_t n, uint64_t *off) {
    const uint8_t *q = (const uint8_t *)p;
    if (q < g_state.heap || q > g_state.heap + g_state.H) return SHMEMG_ERR_NOT_SYMMETRIC;
    uint64_t o = (uint64_t)(q - g_state.heap);
    if (n > g_state.H - o) return SHMEMG_ERR_NOT_SYMMETRIC;
    *off = o;
    return SHMEMG_SUCCESS;
}

int check_pe(int pe) { return (pe >= 0 && pe < g_state.npes) ? SHMEMG_SUCCESS : SHMEMG_ERR_INVALID_ARG; }

int team_get(shmemg_team_t t, HostTeam *out) {
    if (t < 0 || t >= (int)g_state.teams.size() || !g_state.teams[t].valid) return SHMEMG_ERR_INVALID_ARG;
    *out = g_state.teams[t];
    return SHMEMG_SUCCESS;
}

uint64_t balanced_grid(uint64_t nitems, uint64_t cap, int ngroups) {
    if (ngroups > 1) cap = cap / (uint64_t)ngroups > 0 ? cap / (uint64_t)ngroups : 1;
    if (nitems <= cap) return nitems > 0 ? nitems : 1;
    const uint64_t rounds = (nitems + cap - 1) / cap;
    return (nitems + rounds - 1) / rounds;
}

int ctas_for(const void *kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<std::string, int> cache;
    char key[96];
    snprintf(key, sizeof(key), "%p/%d/%zu/%d", kernel, threads, smem, g_state.device);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int n = per_sm * (g_state.sm_count > 0 ? g_state.sm_count : 1);
    cache[key] = n;
    return n;
}

// barrier slots ------------------------------------------------------------------
static int bar_alloc(int count) {
    for (auto it = g_state.bar_free.begin(); it != g_state.bar_free.end(); ++it) {
        if (it->second >= count) {
            int base = it->first, left = it->second - count;
            g_state.bar_free.erase(it);
            if (left) g_state.bar_free[base + count] = left;
            return base;
        }
    }
    return -1;
}
static void bar_release(int base, int count) {
    if (count <= 0) return;
    g_state.bar_free[base] = count;
    // coalesce neighbours
    auto it = g_state.bar_free.find(base);
    if (it != g_state.bar_free.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            g_state.bar_free.erase(it);
            it = prev;
        }
    }
    auto next = std::next(it);
    if (next != g_state.bar_free.end() && it->first + it->second == next->first) {
        it->second += next->second;
        g_state.bar_free.erase(next);
    }
}

static int team_publish(int idx) {
    const HostTeam &h = g_state.teams[idx];
    shmemg_dteam_t d;
    memset(&d, 0, sizeof(d));
    d.start = h.start;
    d.stride = h.stride;
    d.size = h.size;
    d.ngroups = h.ngroups;
    d.gstride = h.gstride;
    d.bar_base = h.bar_base;
    d.valid = h.valid ? 1 : 0;
    uint8_t *dst = g_state.base + SHMEMG_TEAMS_OFF + (uint64_t)idx * sizeof(shmemg_dteam_t);
    int rc = cuda_rc(cudaMemcpy(dst, &d, sizeof(d), cudaMemcpyHostToDevice));
    if (rc) return rc;
    if (h.valid && h.nbar > 0)
        rc = cuda_rc(cudaMemset(g_state.base + SHMEMG_BARRIERS_OFF + (uint64_t)h.bar_base * sizeof(shmemg_dbar_t), 0,
                                (uint64_t)h.nbar * sizeof(shmemg_dbar_t)));
    return rc;
}

static int team_add(const HostTeam &t0, shmemg_team_t *out) {
    HostTeam t = t0;
    int bar = bar_alloc(t.ngroups);
    if (bar < 0) return SHMEMG_ERR_OUT_OF_HEAP;
    t.bar_base = bar;
    t.nbar = t.ngroups;
    t.valid = true;
    int idx = -1;
    for (int i = 2; i < (int)g_state.teams.size(); i++)
        if (!g_state.teams[i].valid) { idx = i; break; }
    if (idx < 0) {
        if ((int)g_state.teams.size() >= SHMEMG_MAX_TEAMS) { bar_release(bar, t.nbar); return SHMEMG_ERR_OUT_OF_HEAP; }
        idx = (int)g_state.teams.size();
        g_state.teams.push_back(HostTeam());
    }
    g_state.teams[idx] = t;
    int rc = team_publish(idx);
    if (rc) { g_state.teams[idx].valid = false; bar_release(bar, t.nbar); return rc; }
    *out = idx;
    return SHMEMG_SUCCESS;
}

}  // namespace shmemg

using namespace shmemg;

// ================================================================== C ABI
extern "C" {

int shmemg_required_heap_bytes(int npes, uint64_t H, uint64_t *out) {
    if (!out || npes < 1 || H < 256 || (H & 255)) return SHMEMG_ERR_INVALID_ARG;
    if (H > (UINT64_MAX - SHMEMG_RESERVED_BYTES) / (uint64_t)npes) return SHMEMG_ERR_INVALID_ARG;
    *out = SHMEMG_RESERVED_BYTES + (uint64_t)npes * H;
    return SHMEMG_SUCCESS;
}

int shmemg_init(const shmemg_init_attr_t *a) {
    State &s = st();
    if (s.init) return SHMEMG_ERR_BUSY;
    if (!a || !a->heap_ptr || ((uintptr_t)a->heap_ptr & 255)) return SHMEMG_ERR_INVALID_ARG;
    if (a->pe_mode != SHMEMG_PE_MODE_CTA && a->pe_mode != SHMEMG_PE_MODE_CLUSTER) return SHMEMG_ERR_INVALID_ARG;
    int cd = a->cluster_dim <= 0 ? 1 : a->cluster_dim;
    if (cd > 8 || (cd & (cd - 1))) return SHMEMG_ERR_INVALID_ARG;
    if (a->pe_mode == SHMEMG_PE_MODE_CTA && a->npes % cd) return SHMEMG_ERR_INVALID_ARG;
    uint64_t need = 0;
    int rc = shmemg_required_heap_bytes(a->npes, a->heap_bytes_per_pe, &need);
    if (rc) return rc;
    if (a->heap_bytes < need) return SHMEMG_ERR_INVALID_ARG;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, a->heap_ptr) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return SHMEMG_ERR_INVALID_ARG;  // the heap must be device memory (Sec. 6.1 memory type)
    }
    int dev = 0;
    if ((rc = cuda_rc(cudaGetDevice(&dev)))) return rc;
    if (pa.device != dev) return SHMEMG_ERR_INVALID_ARG;
    s = State();
    s.device = dev;
    cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
    s.npes = a->npes;
    s.pe_mode = a->pe_mode;
    s.cluster_dim = cd;
    s.H = a->heap_bytes_per_pe;
    s.base = (uint8_t *)a->heap_ptr;
    s.heap = s.base + SHMEMG_RESERVED_BYTES;
    s.heap_bytes = a->heap_bytes;
    s.timeout_ns = a->wait_timeout_ns ? a->wait_timeout_ns : 2000000000ull;
    const char *env = getenv("SHMEMG_WAIT_TIMEOUT_NS");
    if (env && *env) s.timeout_ns = strtoull(env, nullptr, 10);
    s.free_ranges[0] = s.H;
    s.bar_free[0] = SHMEMG_MAX_BARRIERS;
    cudaStream_t strm = to_stream(a->stream);
    if ((rc = cuda_rc(cudaMemsetAsync(s.base, 0, SHMEMG_RESERVED_BYTES, strm)))) return rc;
    if ((rc = cuda_rc(cudaStreamSynchronize(strm)))) return rc;
    s.init = true;
    // WORLD: every PE; SHARED: the PEs of one cluster (CTA mode), else the PE itself
    HostTeam w;
    w.start = 0; w.stride = 1; w.size = s.npes; w.ngroups = 1; w.gstride = 0;
    HostTeam sh;
    int shsize = (s.pe_mode == SHMEMG_PE_MODE_CTA) ? cd : 1;
    sh.start = 0; sh.stride = 1; sh.size = shsize; sh.ngroups = s.npes / shsize; sh.gstride = shsize;
    s.teams.resize(2);
    for (int i = 0; i < 2; i++) {
        HostTeam t = i == 0 ? w : sh;
        int bar = bar_alloc(t.ngroups);
        t.bar_base = bar;
        t.nbar = t.ngroups;
        t.valid = true;
        s.teams[i] = t;
        if ((rc = team_publish(i))) { s.init = false; return rc; }
    }
    return SHMEMG_SUCCESS;
}

int shmemg_finalize(void) {
    State &s = st();
    if (!s.init) return SHMEMG_ERR_NOT_INITIALIZED;
    int rc = cuda_rc(cudaDeviceSynchronize());
    s = State();
    return rc;
}

int shmemg_initialized(int *out) {
    if (!out) return SHMEMG_ERR_INVALID_ARG;
    *out = st().init ? 1 : 0;
    return SHMEMG_SUCCESS;
}

int shmemg_n_pes(int *out) {
    if (int rc = check_init()) return rc;
    if (!out) return SHMEMG_ERR_INVALID_ARG;
    *out = st().npes;
    return SHMEMG_SUCCESS;
}

int shmemg_device_ctx(shmemg_device_ctx_t *out) {
    if (int rc = check_init()) return rc;
    if (!out) return SHMEMG_ERR_INVALID_ARG;
    *out = device_ctx();
    return SHMEMG_SUCCESS;
}

// --------------------------------------------------------------- allocation
int shmemg_malloc(uint64_t bytes, void **out) {
    if (int rc = check_init()) return rc;
    if (!out) return SHMEMG_ERR_INVALID_ARG;
    State &s = st();
    uint64_t need = bytes ? (bytes + 255) & ~255ull : 256;
    for (auto it = s.free_ranges.begin(); it != s.free_ranges.end(); ++it) {
        if (it->second >= need) {
            uint64_t off = it->first, left = it->second - need;
            s.free_ranges.erase(it);
            if (left) s.free_ranges[off + need] = left;
            s.live[off] = need;
            *out = s.heap + off;
            return SHMEMG_SUCCESS;
        }
    }
    return SHMEMG_ERR_OUT_OF_HEAP;
}

int shmemg_calloc(uint64_t bytes, void **out, void *stream) {
    int rc = shmemg_malloc(bytes, out);
    if (rc) return rc;
    State &s = st();
    uint64_t off = (uint64_t)((uint8_t *)*out - s.heap);
    uint64_t len = s.live[off];
    for (int p = 0; p < s.npes; p++) {
        if ((rc = cuda_rc(cudaMemsetAsync(s.heap + (uint64_t)p * s.H + off, 0, len, to_stream(stream))))) return rc;
    }
    return SHMEMG_SUCCESS;
}

int shmemg_free(void *ptr) {
    if (int rc = check_init()) return rc;
    if (!ptr) return SHMEMG_SUCCESS;
    State &s = st();
    uint64_t off = 0;
    if (sym_offset(ptr, 0, &off)) return SHMEMG_ERR_NOT_SYMMETRIC;
    auto it = s.live.find(off);
    if (it == s.live.end()) return SHMEMG_ERR_NOT_SYMMETRIC;
    uint64_t len = it->second;
    s.live.erase(it);
    s.free_ranges[off] = len;
    auto f = s.free_ranges.find(off);
    if (f != s.free_ranges.begin()) {
        auto prev = std::prev(f);
        if (prev->first + prev->second == f->first) {
            prev->second += f->second;
            s.free_ranges.erase(f);
            f = prev;
        }
    }
    auto next = std::next(f);
    if (next != s.free_ranges.end() && f->first + f->second == next->first) {
        f->second += next->second;
        s.free_ranges.erase(next);
    }
    return SHMEMG_SUCCESS;
}

int shmemg_ptr(const void *sym, int pe, void **out) {
    if (int rc = check_init()) return rc;
    if (!out) return SHMEMG_ERR_INVALID_ARG;
    if (check_pe(pe)) return SHMEMG_ERR_INVALID_ARG;
    uint64_t off;
    if (sym_offset(sym, 0, &off)) return SHMEMG_ERR_NOT_SYMMETRIC;
    *out = st().heap + (uint64_t)pe * st().H + off;
    return SHMEMG_SUCCESS;
}

// --------------------------------------------------------------- teams
int shmemg_team_split_strided(shmemg_team_t parent, int start, int stride, int size, shmemg_team_t *out) {
    if (int rc = check_init()) return rc;
    if (!out) return SHMEMG_ERR_INVALID_ARG;
    *out = SHMEMG_TEAM_INVALID;
    HostTeam p;
    if (team_get(parent, &p)) return SHMEMG_ERR_INVALID_ARG;
    if (p.ngroups != 1) return SHMEMG_ERR_UNSUPPORTED;
    if (size < 1 || stride < 1 || start < 0 || start + (int64_t)(size - 1) * stride >= p.size) return SHMEMG_ERR_INVALID_ARG;
    HostTeam t;
    t.start = p.start + start * p.stride;
    t.stride = stride * p.stride;
    t.size = size;
    t.ngroups = 1;
    t.gstride = 0;
    return team_add(t, out);
}

int shmemg_team_destroy(shmemg_team_t team) {
    if (int rc = check_init()) return rc;
    if (team == SHMEMG_TEAM_WORLD || team == SHMEMG_TEAM_SHARED) return SHMEMG_ERR_INVALID_ARG;
    HostTeam t;
    if (team_get(team, &t)) return SHMEMG_ERR_INVALID_ARG;
    bar_release(t.bar_base, t.nbar);
    st().teams[team].valid = false;
    return team_publish(team);
}

int shmemg_team_n_pes(shmemg_team_t team, int *out) {
    if (int rc = check_init()) return rc;
    HostTeam t;
    if (!out || team_get(team, &t)) return SHMEMG_ERR_INVALID_ARG;
    *out = t.size;
    return SHMEMG_SUCCESS;
}

static int world_of(const HostTeam &t, int group, int r) { return t.start + group * t.gstride + r * t.stride; }
static int rank_in(const HostTeam &t, int group, int pe) {
    int rel = pe - t.start - group * t.gstride;
    if (rel < 0 || rel % t.stride) return -1;
    int r = rel / t.stride;
    return r < t.size ? r : -1;
}

int shmemg_team_translate_pe(shmemg_team_t src_team, int src_pe, shmemg_team_t dest_team, int *out) {
    if (int rc = check_init()) return rc;
    HostTeam a, b;
    if (!out || team_get(src_team, &a) || team_get(dest_team, &b)) return SHMEMG_ERR_INVALID_ARG;
    *out = -1;
    if (src_pe < 0 || src_pe >= a.size) return SHMEMG_ERR_INVALID_ARG;
    // grouped (SHARED) teams: ranks refer to group 0 unless the other team pins a group
    int w = world_of(a, 0, src_pe);
    int g = b.gstride > 0 ? (w - b.start) / b.gstride : 0;
    if (g < 0 || g >= b.ngroups) return SHMEMG_SUCCESS;
    *out = rank_in(b, g, w);
    return SHMEMG_SUCCESS;
}

// --------------------------------------------------------------- capabilities
int shmemg_query_capabilities(shmemg_team_t team, shmemg_caps_t *out) {
    if (int rc = check_init()) return rc;
    HostTeam t;
    if (!out || team_get(team, &t)) return SHMEMG_ERR_INVALID_ARG;
    State &s = st();
    memset(out, 0, sizeof(*out));
    out->flags = SHMEMG_CAP_GPU_AWARE_HOST | SHMEMG_CAP_DEVICE_RMA | SHMEMG_CAP_DEVICE_AMO | SHMEMG_CAP_DEVICE_SIGNAL |
                 SHMEMG_CAP_DEVICE_COLL | SHMEMG_CAP_STREAM_ORDERED | SHMEMG_CAP_DEVICE_CTX_DEFAULT |
                 SHMEMG_CAP_DEVICE_TEAMS | SHMEMG_CAP_PTR_DEVICE | SHMEMG_CAP_PROGRESS_GPU | SHMEMG_CAP_EXPLICIT_DEVICE_CTX |
                 SHMEMG_CAP_PERSISTENT_SERVER | SHMEMG_CAP_BATCHED_COLL | SHMEMG_CAP_QUANTIZED_REDUCE;
    out->default_heap = SHMEMG_HEAP_GPU;
    out->path = SHMEMG_PATH_DIRECT_LOCAL_HBM;
    // the shared team of a CTA-mode heap is a thread-block cluster: its device-initiated
    // barrier and small collectives go through distributed shared memory
    if (team == SHMEMG_TEAM_SHARED && s.pe_mode == SHMEMG_PE_MODE_CTA && s.cluster_dim > 1) out->path |= SHMEMG_PATH_DSMEM;
    out->rma_scopes = SHMEMG_SCOPE_THREAD | SHMEMG_SCOPE_WARP | SHMEMG_SCOPE_BLOCK | SHMEMG_SCOPE_CLUSTER;
    out->coll_scopes = SHMEMG_SCOPE_WARP | SHMEMG_SCOPE_BLOCK | SHMEMG_SCOPE_CLUSTER | SHMEMG_SCOPE_GRID;
    out->device_ordinal = s.device;
    out->pe_mode = s.pe_mode;
    out->cluster_dim = s.cluster_dim;
    out->team_n_pes = t.size;
    out->shared_team_size = s.teams[SHMEMG_TEAM_SHARED].size;
    out->device_ctx_count = SHMEMG_DEVICE_CTX_COUNT;
    out->heap_bytes_per_pe = s.H;
    uint64_t best = 0;
    for (auto &f : s.free_ranges) best = f.second > best ? f.second : best;
    out->heap_free_bytes = best;
    out->wait_timeout_ns = s.timeout_ns;
    return SHMEMG_SUCCESS;
}

// --------------------------------------------------------------- status
int shmemg_get_status(int *code, int64_t *detail) {
    if (int rc = check_init()) return rc;
    int rc = cuda_rc(cudaDeviceSynchronize());
    if (rc) return rc;
    struct { int32_t code, pad; int64_t detail; } w;
    if ((rc = cuda_rc(cudaMemcpy(&w, st().base + SHMEMG_STATUS_OFF, sizeof(w), cudaMemcpyDeviceToHost)))) return rc;
    if (code) *code = w.code;
    if (detail) *detail = w.detail;
    return SHMEMG_SUCCESS;
}

int shmemg_clear_status(void *stream) {
    if (int rc = check_init()) return rc;
    return cuda_rc(cudaMemsetAsync(st().base + SHMEMG_STATUS_OFF, 0, 16, to_stream(stream)));
}

const char *shmemg_strerror(int code) {
    switch (code) {
    case SHMEMG_SUCCESS: return "success";
    case SHMEMG_ERR_INVALID_ARG: return "invalid argument";
    case SHMEMG_ERR_NOT_INITIALIZED: return "not initialized";
    case SHMEMG_ERR_OUT_OF_HEAP: return "out of symmetric heap";
    case SHMEMG_ERR_NOT_SYMMETRIC: return "pointer or range not in the symmetric heap";
    case SHMEMG_ERR_UNSUPPORTED: return "unsupported";
    case SHMEMG_ERR_TIMEOUT: return "device wait timed out";
    case SHMEMG_ERR_CUDA: return g_cuda_msg.empty() ? "CUDA error" : g_cuda_msg.c_str();
    case SHMEMG_ERR_BUSY: return "busy";
    case SHMEMG_ERR_DEVICE: return "device-side error";
    default: return "unknown error";
    }
}

// --------------------------------------------------------------- ordering
static __global__ void k_fence() { shmemg_d_fence_sys(); }

int shmemg_fence(void *stream) {
    if (int rc = check_init()) return rc;
    k_fence<<<1, 1, 0, to_stream(stream)>>>();
    return cuda_rc(cudaGetLastError());
}

int shmemg_quiet(void *stream) {
    if (int rc = check_init()) return rc;
    return cuda_rc(cudaStreamSynchronize(to_stream(stream)));
}

int shmemg_barrier_all(void *stream) {
    if (int rc = check_init()) return rc;
    return cuda_rc(cudaStreamSynchronize(to_stream(stream)));
}

int shmemg_team_sync(shmemg_team_t team, void *stream) {
    if (int rc = check_init()) return rc;
    HostTeam t;
    if (team_get(team, &t)) return SHMEMG_ERR_INVALID_ARG;
    // every member PE is driven by this host thread through `stream`: stream order is
    // the team barrier; enqueue a device fence so the barrier also orders memory
    k_fence<<<1, 1, 0, to_stream(stream)>>>();
    return cuda_rc(cudaGetLastError());
}

}  // extern "C"
