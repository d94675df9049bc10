// Library-internal host state shared by the translation units of libshmemg.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <vector>

#include "shmemg.h"
#include "shmemg_device.cuh"

namespace shmemg {

struct HostTeam {
    int32_t start = 0, stride = 1, size = 0, ngroups = 1, gstride = 0;
    int32_t bar_base = 0, nbar = 0;
    bool valid = false;
};

struct State {
    bool init = false;
    int npes = 0, pe_mode = 0, cluster_dim = 1;
    uint64_t H = 0;
    uint8_t *base = nullptr;   // caller's allocation (reserved prefix first)
    uint8_t *heap = nullptr;   // PE 0's partition
    uint64_t heap_bytes = 0;
    uint64_t timeout_ns = 0;
    int device = 0, sm_count = 0;
    // symmetric allocator: free ranges and live objects (offset -> bytes)
    std::map<uint64_t, uint64_t> free_ranges, live;
    std::vector<HostTeam> teams;
    std::map<int32_t, int32_t> bar_free;  // barrier slot ranges: base -> count
    uint64_t call_seq = 0;               // rotates scratch slots of multi-CTA signal puts
};

State &st();
shmemg_device_ctx_t device_ctx();

// --- argument helpers (return SHMEMG_* codes)
int check_init();
// canonical symmetric pointer + length -> offset; SHMEMG_ERR_NOT_SYMMETRIC if outside
int sym_offset(const void *p, uint64_t n, uint64_t *off);
int check_pe(int pe);
int team_get(shmemg_team_t t, HostTeam *out);
inline cudaStream_t to_stream(void *s) { return (cudaStream_t)s; }
int cuda_rc(cudaError_t e);  // maps a CUDA error to SHMEMG_ERR_CUDA (records the message)

// max co-resident CTAs of a kernel (occupancy), cached per kernel
int ctas_for(const void *kernel, int threads, size_t smem);
// Grid for `nitems` equal work items taken grid-stride by at most `cap` resident CTAs
// (split over `ngroups` grid rows): as many rounds as the items need, and the fewest CTAs
// that finish them in that many rounds, so no partial last wave runs on an idle GPU.
uint64_t balanced_grid(uint64_t nitems, uint64_t cap, int ngroups = 1);

// cooperative launch with one CTA per PE (pe_mode CTA) or one cluster of cluster_dim CTAs
// per PE, `threads` per CTA (0: the interpreter's count), the grid grid_mult times that
// (the interpreter's context agents: CTA npes + p serves PE p); SHMEMG_ERR_UNSUPPORTED if
// the GPU cannot hold every CTA at once
int launch_pe_grid(const void *kernel, void **args, size_t smem, cudaStream_t s, int threads = 0, int grid_mult = 1);
int interp_threads();

// splitmix64 (Steele, Lea, Flood, OOPSLA 2014): first output of the stream started at
// state seed ^ i -- the counter-based draw of the AMO stream and of staged payloads.
__device__ __forceinline__ uint64_t cb64(uint64_t seed, uint64_t i) {
    uint64_t z = (seed ^ i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// scratch words in the reserved prefix: [SHMEMG_SCRATCH_OFF, +2 MiB)
enum : uint64_t {
    SCR_SIGNAL_DONE = 0,            // 4096 uint32 counters for multi-CTA put_signal
    SCR_SIGNAL_DONE_SLOTS = 4096,
    SCR_WORK = 64 << 10,            // work counters of persistent kernels (uint64 each)
};

}  // namespace shmemg
