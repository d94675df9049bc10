/*
 * shmemg.h -- C ABI of a GPU-aware OpenSHMEM symmetric heap on one GPU.
 *
 * Model (paper "Toward a Unified GPU-Aware OpenSHMEM Specification"):
 *  - Sec. 2.1: each processing element (PE) exposes a symmetric heap of the same size
 *    and allocation order, so a remote address is computable from a local one.
 *  - Sec. 6.1: one GPU symmetric heap, created at initialisation, from which
 *    shmemg_malloc allocates symmetric objects; traits are size and memory type.
 *  - Sec. 6.2: a host default context and a device default context
 *    (SHMEM_DEVICE_CTX_DEFAULT) published to the device; device teams WORLD/SHARED.
 *  - Sec. 6.3: host-executed, stream-triggered and device-initiated operations;
 *    blocking operations complete locally, _nbi ones at quiet; atomicity does not
 *    imply ordering; collectives need uniform participation.
 *  - Sec. 6.4: fence orders, quiet completes; the host needs stream synchronisation
 *    to see device results (Fig. 3).
 *  - Sec. 6.5: per-team capability queries, locality and path reporting.
 *
 * Here one GPU's HBM holds npes *virtual PEs*: npes equal partitions of H bytes of a
 * single device allocation that the CALLER owns (this library never allocates the
 * heap).  A PE is a thread block (pe_mode CTA) or a thread-block cluster (pe_mode
 * CLUSTER) of the kernels that run device-initiated work.
 *
 * Conventions for every function below:
 *  - Return value: SHMEMG_SUCCESS (0) or a negative SHMEMG_ERR_* code.  Argument checks
 *    happen on the host before anything is launched; a failed check launches nothing.
 *  - Symmetric pointers are *canonical*: addresses inside PE 0's partition, as returned
 *    by shmemg_malloc.  The PE is a separate argument.  A pointer or byte range outside
 *    [partition base, partition base + H) gives SHMEMG_ERR_NOT_SYMMETRIC.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).  Host
 *    operations are stream-triggered: they are enqueued on the stream and return
 *    without waiting; shmemg_quiet(stream) waits for them (Sec. 6.4 quiet table).
 *  - Device buffers that are not symmetric (fetched-value arrays, op lists, timing
 *    arrays) are plain device pointers owned by the caller.
 *  - Errors found by device code (wait timeouts, device bounds checks) are recorded in
 *    a device status word; read it with shmemg_get_status.  Device waits are bounded
 *    by the init attribute wait_timeout_ns.
 *  - The library keeps one global state: calls are not thread-safe with respect to
 *    each other (one host thread speaks for all virtual PEs).
 */
#ifndef SHMEMG_H
#define SHMEMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status codes */
#define SHMEMG_SUCCESS 0
#define SHMEMG_ERR_INVALID_ARG (-1)
#define SHMEMG_ERR_NOT_INITIALIZED (-2)
#define SHMEMG_ERR_OUT_OF_HEAP (-3)
#define SHMEMG_ERR_NOT_SYMMETRIC (-4)
#define SHMEMG_ERR_UNSUPPORTED (-5)
#define SHMEMG_ERR_TIMEOUT (-6)
#define SHMEMG_ERR_CUDA (-7)
#define SHMEMG_ERR_BUSY (-8)
#define SHMEMG_ERR_DEVICE (-9)

/* ----------------------------------------------------------------- enums */
enum { SHMEMG_PE_MODE_CTA = 0, SHMEMG_PE_MODE_CLUSTER = 1 };
enum { SHMEMG_INT32 = 0, SHMEMG_INT64 = 1, SHMEMG_FLOAT = 2, SHMEMG_UINT64 = 3 };
enum { SHMEMG_SUM = 0, SHMEMG_MAX = 1, SHMEMG_MIN = 2 };
enum { SHMEMG_SIGNAL_SET = 0, SHMEMG_SIGNAL_ADD = 1 };
enum { SHMEMG_CMP_EQ = 0, SHMEMG_CMP_NE, SHMEMG_CMP_GT, SHMEMG_CMP_GE, SHMEMG_CMP_LT, SHMEMG_CMP_LE };
enum { SHMEMG_FMT_BF16 = 0, SHMEMG_FMT_E4M3 = 1 };

/* Teams (Sec. 6.2 device teams; OpenSHMEM 1.6 teams).  WORLD = all PEs.  SHARED =
 * the PEs of the caller's GPU locality domain below the whole HBM: the thread-block
 * cluster (pe_mode CTA, cluster_dim PEs per cluster), so a host collective on SHARED
 * runs once per cluster group; with pe_mode CLUSTER or cluster_dim 1 it is the PE
 * itself.  The device teams have the same membership as the host teams here, and
 * host and device operations share one atomicity domain (the GPU's L2). */
typedef int32_t shmemg_team_t;
#define SHMEMG_TEAM_INVALID (-1)
#define SHMEMG_TEAM_WORLD 0
#define SHMEMG_TEAM_SHARED 1
#define SHMEMG_DEVICE_TEAM_WORLD SHMEMG_TEAM_WORLD
#define SHMEMG_DEVICE_TEAM_SHARED SHMEMG_TEAM_SHARED
#define SHMEMG_MAX_TEAMS 4096

/* Reserved device bytes in front of the partitions: status word, team table, team
 * barrier words, scratch counters.  Partition p starts at heap_ptr + RESERVED + p*H. */
#define SHMEMG_RESERVED_BYTES (4u << 20)

/* ----------------------------------------------------------------- init */
typedef struct {
    int32_t npes;                /* number of virtual PEs, >= 1 */
    int32_t pe_mode;             /* SHMEMG_PE_MODE_CTA or _CLUSTER */
    int32_t cluster_dim;         /* CTAs per cluster, 1..8 (CLUSTER: CTAs per PE) */
    int32_t reserved0;
    uint64_t heap_bytes_per_pe;  /* H: multiple of 256, >= 256 */
    void *heap_ptr;              /* device pointer, 256-byte aligned, caller-owned */
    uint64_t heap_bytes;         /* >= shmemg_required_heap_bytes(npes, H) */
    void *stream;                /* stream used for initialisation work */
    uint64_t wait_timeout_ns;    /* bound of every device wait; 0 = 2 s */
} shmemg_init_attr_t;

/* Bytes the caller must allocate for npes partitions of H bytes (reserved prefix
 * included).  Sec. 6.1: the GPU heap is static and created at initialisation. */
int shmemg_required_heap_bytes(int npes, uint64_t heap_bytes_per_pe, uint64_t *out);

/* Initialise on the current CUDA device: carves the caller's allocation into npes
 * partitions, builds WORLD and SHARED, zeroes the reserved prefix on attr->stream and
 * waits for it, and publishes the device default context.  Fig. 6 (context
 * lifecycle): init -> publish device-visible handle -> kernel use -> finalize.
 * SHMEMG_ERR_BUSY if already initialised. */
int shmemg_init(const shmemg_init_attr_t *attr);
/* Synchronises the device, drops teams, allocations and batches.  The heap memory
 * stays the caller's. */
int shmemg_finalize(void);
int shmemg_initialized(int *out);
int shmemg_n_pes(int *out);

/* Device default context (SHMEM_DEVICE_CTX_DEFAULT, Sec. 6.2): the values device code
 * needs to address the heap, passed to kernels by value. */
typedef struct {
    uint8_t *heap;          /* base of PE 0's partition (device address) */
    uint64_t pe_stride;     /* H */
    int32_t npes;
    int32_t pe_mode;
    int32_t cluster_dim;
    int32_t reserved0;
    uint8_t *state;         /* reserved prefix (device address) */
    uint64_t timeout_ns;
} shmemg_device_ctx_t;
int shmemg_device_ctx(shmemg_device_ctx_t *out);

/* ----------------------------------------------------------------- allocation */
/* Symmetric allocation (Sec. 6.1 shmemg_malloc): the same offset in every partition,
 * 256-byte aligned.  Collective by construction (one host thread speaks for all PEs).
 * *out = canonical pointer (inside PE 0's partition).  SHMEMG_ERR_OUT_OF_HEAP if no
 * free range of that size is left. */
int shmemg_malloc(uint64_t bytes, void **out);
/* shmemg_malloc followed by a zero fill of the object on every PE, on stream. */
int shmemg_calloc(uint64_t bytes, void **out, void *stream);
/* Frees an object returned by shmemg_malloc/calloc; NULL is a no-op; anything else
 * gives SHMEMG_ERR_NOT_SYMMETRIC. */
int shmemg_free(void *ptr);
/* Device address of the symmetric object `sym` on PE `pe` (shmem_ptr analogue,
 * Sec. 6.3 pointer queries).  Access domain: DEVICE ONLY -- never dereference it on
 * the host (capabilities report PTR_DEVICE, not PTR_HOST). */
int shmemg_ptr(const void *sym, int pe, void **out_device_ptr);

/* ----------------------------------------------------------------- teams */
/* New team of `size` PEs of `parent`: parent ranks start, start+stride, ... (OpenSHMEM
 * 1.6 team split).  SHARED cannot be split (SHMEMG_ERR_UNSUPPORTED). */
int shmemg_team_split_strided(shmemg_team_t parent, int start, int stride, int size,
                              shmemg_team_t *out);
int shmemg_team_destroy(shmemg_team_t team);
int shmemg_team_n_pes(shmemg_team_t team, int *out);
/* PE number in dest_team of rank src_pe of src_team, or -1 if not a member.  For
 * SHARED, ranks refer to the group that contains world PE `src_pe`'s cluster. */
int shmemg_team_translate_pe(shmemg_team_t src_team, int src_pe, shmemg_team_t dest_team,
                             int *out);

/* ----------------------------------------------------------------- capabilities */
/* Sec. 6.5: per-team capability query.  Flags distinguish GPU-aware host-initiated
 * support from device-initiated APIs and report stream-ordered variants separately. */
#define SHMEMG_CAP_GPU_AWARE_HOST (1ull << 0)      /* host ops on GPU symmetric data */
#define SHMEMG_CAP_DEVICE_RMA (1ull << 1)
#define SHMEMG_CAP_DEVICE_AMO (1ull << 2)
#define SHMEMG_CAP_DEVICE_SIGNAL (1ull << 3)
#define SHMEMG_CAP_DEVICE_COLL (1ull << 4)
#define SHMEMG_CAP_STREAM_ORDERED (1ull << 5)      /* host ops take a stream */
#define SHMEMG_CAP_DEVICE_CTX_DEFAULT (1ull << 6)
#define SHMEMG_CAP_EXPLICIT_DEVICE_CTX (1ull << 7) /* explicit device contexts (script ops) */
#define SHMEMG_CAP_DEVICE_TEAMS (1ull << 8)
#define SHMEMG_CAP_PTR_DEVICE (1ull << 9)          /* shmemg_ptr valid in device code */
#define SHMEMG_CAP_PTR_HOST (1ull << 10)           /* not provided */
#define SHMEMG_CAP_PROGRESS_GPU (1ull << 11)       /* device ops need no host progress */
#define SHMEMG_CAP_HOST_PROGRESS_REQUIRED (1ull << 12) /* not set */
#define SHMEMG_CAP_MIXED_HOST_DEVICE_COLL (1ull << 13) /* not set: mixing is undefined */
#define SHMEMG_CAP_PERSISTENT_SERVER (1ull << 14)
#define SHMEMG_CAP_BATCHED_COLL (1ull << 15)
#define SHMEMG_CAP_QUANTIZED_REDUCE (1ull << 16)

enum { SHMEMG_HEAP_GPU = 1 };
enum { SHMEMG_PATH_DIRECT_LOCAL_HBM = 1, SHMEMG_PATH_DSMEM = 2 };
enum { SHMEMG_SCOPE_THREAD = 1, SHMEMG_SCOPE_WARP = 2, SHMEMG_SCOPE_BLOCK = 4,
       SHMEMG_SCOPE_CLUSTER = 8, SHMEMG_SCOPE_GRID = 16 };

typedef struct {
    uint64_t flags;             /* SHMEMG_CAP_* */
    int32_t default_heap;       /* SHMEMG_HEAP_GPU: the only heap is GPU-attached */
    int32_t path;               /* bitmask of SHMEMG_PATH_* used for device-initiated ops */
    uint32_t rma_scopes;        /* SHMEMG_SCOPE_* supported by device RMA */
    uint32_t coll_scopes;       /* SHMEMG_SCOPE_* supported by device collectives */
    int32_t device_ordinal;     /* every PE of every team lives on this GPU */
    int32_t pe_mode;
    int32_t cluster_dim;
    int32_t team_n_pes;
    int32_t shared_team_size;   /* PEs in the caller's device shared team (locality) */
    int32_t device_ctx_count;   /* device contexts per PE: the default + explicit ones */
    uint64_t heap_bytes_per_pe;
    uint64_t heap_free_bytes;   /* largest free symmetric range */
    uint64_t wait_timeout_ns;
} shmemg_caps_t;
int shmemg_query_capabilities(shmemg_team_t team, shmemg_caps_t *out);

/* ----------------------------------------------------------------- status */
/* Device status word: first error recorded by device code since the last clear
 * (SHMEMG_SUCCESS if none) and an operation-specific detail (op index, PE ...).
 * For SHMEMG_ERR_TIMEOUT of a bulk (TMA) ring: -2 a device-initiated copy, -3 a
 * host-issued bulk transfer or an explicit context's queue, each after the loads still
 * in flight have landed; -4 a load that did not land even then (the launch's results are
 * void and the ring was not used again); -5 a context agent that saw no post, no progress
 * of its PE and no end of the script for 8 x the wait timeout and left (a quiet on its
 * contexts then times out with the op index as detail).  Synchronises the device. */
int shmemg_get_status(int *code, int64_t *detail);
int shmemg_clear_status(void *stream);
const char *shmemg_strerror(int code);

/* ----------------------------------------------------------------- host RMA */
/* Sec. 2.1 put: bytes [src, src+n) of PE `issuer` -> [dst, dst+n) of PE `pe`.
 * Stream-triggered; blocking and _nbi forms have the same stream-ordered semantics
 * (the source may be reused by any later operation on the stream); completion for the
 * host is shmemg_quiet(stream).  Overlapping source and destination ranges are
 * undefined. */
int shmemg_putmem(void *dst, const void *src, uint64_t n, int pe, int issuer, void *stream);
int shmemg_putmem_nbi(void *dst, const void *src, uint64_t n, int pe, int issuer, void *stream);
/* Sec. 2.1 get: bytes [src, src+n) of PE `pe` -> [dst, dst+n) of PE `issuer`. */
int shmemg_getmem(void *dst, const void *src, uint64_t n, int pe, int issuer, void *stream);
int shmemg_getmem_nbi(void *dst, const void *src, uint64_t n, int pe, int issuer, void *stream);

/* ----------------------------------------------------------------- host AMOs */
/* Sec. 2.1 atomics on a symmetric word of PE `pe`.  fetch_add / fetch_xor return the
 * old value and store old+v (wrapping) / old^v; compare_swap returns the old value and
 * stores v iff old == cond.  The old value is written to the caller's device pointer
 * `fetched` (may be NULL).  Sec. 6.3: atomicity does not imply ordering. */
int shmemg_int64_atomic_fetch_add(int64_t *target, int64_t v, int pe, int64_t *fetched, void *stream);
int shmemg_int64_atomic_compare_swap(int64_t *target, int64_t cond, int64_t v, int pe,
                                     int64_t *fetched, void *stream);
int shmemg_int64_atomic_fetch_xor(int64_t *target, int64_t v, int pe, int64_t *fetched, void *stream);
int shmemg_int32_atomic_fetch_add(int32_t *target, int32_t v, int pe, int32_t *fetched, void *stream);
int shmemg_int32_atomic_compare_swap(int32_t *target, int32_t cond, int32_t v, int pe,
                                     int32_t *fetched, void *stream);
int shmemg_int32_atomic_fetch_xor(int32_t *target, int32_t v, int pe, int32_t *fetched, void *stream);

/* ----------------------------------------------------------------- signals */
/* Sec. 7 (put-signal): the put, then the uint64 signal word `sig` (symmetric, on PE
 * `pe`) is set to / incremented by `sigval` (SHMEMG_SIGNAL_SET / _ADD) after the data
 * is written.  Signal and target must be in the GPU symmetric heap. */
int shmemg_putmem_signal(void *dst, const void *src, uint64_t n, uint64_t *sig, uint64_t sigval,
                         int sig_op, int pe, int issuer, void *stream);
/* Stream-ordered wait: later work on `stream` starts once "sig(on pe) cmp value" holds
 * (unsigned compare).  Bounded by wait_timeout_ns: on timeout the status word records
 * SHMEMG_ERR_TIMEOUT and the stream continues. */
int shmemg_signal_wait_until(uint64_t *sig, int pe, int cmp, uint64_t value, void *stream);

/* ----------------------------------------------------------------- ordering */
/* Sec. 6.4.  fence: orders later operations on `stream` after earlier ones (stream
 * order already does; enqueues a device fence).  quiet: the host waits until every
 * operation enqueued on `stream` is complete and visible (host quiet = completion +
 * stream synchronisation).  barrier_all / team_sync: stream-ordered barriers of all
 * PEs / the team's PEs (all PEs are driven by this host thread, so stream order is the
 * barrier); barrier_all also completes outstanding operations on the stream like
 * quiet does. */
int shmemg_fence(void *stream);
int shmemg_quiet(void *stream);
int shmemg_barrier_all(void *stream);
int shmemg_team_sync(shmemg_team_t team, void *stream);

/* ----------------------------------------------------------------- host collectives */
/* OpenSHMEM 1.6 team collectives (inherited unchanged, Sec. 6.3), executed by one
 * full-grid kernel on `stream`.  All buffers are symmetric objects.
 * broadcast: every member's dst (the root's too) receives root's src; root = team rank.
 * fcollect: every member's dst = the members' src blocks (n bytes each) in rank order.
 * alltoall: member j's dst block i = member i's src block j (blocks of n bytes).
 * reduce: all-reduce; every member's dst[k] = op over members of src[k]; integer sums
 * wrap; float sums use the fixed rank-pairwise tree (bitwise reproducible); dst == src
 * is allowed (in place), other overlaps are undefined. */
int shmemg_broadcastmem(shmemg_team_t team, void *dst, const void *src, uint64_t n, int root,
                        void *stream);
int shmemg_fcollectmem(shmemg_team_t team, void *dst, const void *src, uint64_t n, void *stream);
int shmemg_alltoallmem(shmemg_team_t team, void *dst, const void *src, uint64_t n, void *stream);
int shmemg_reduce(shmemg_team_t team, void *dst, const void *src, uint64_t nelems, int dtype,
                  int op, void *stream);
int shmemg_int32_sum_reduce(shmemg_team_t team, int32_t *dst, const int32_t *src, uint64_t n, void *stream);
int shmemg_int32_max_reduce(shmemg_team_t team, int32_t *dst, const int32_t *src, uint64_t n, void *stream);
int shmemg_int32_min_reduce(shmemg_team_t team, int32_t *dst, const int32_t *src, uint64_t n, void *stream);
int shmemg_int64_sum_reduce(shmemg_team_t team, int64_t *dst, const int64_t *src, uint64_t n, void *stream);
int shmemg_int64_max_reduce(shmemg_team_t team, int64_t *dst, const int64_t *src, uint64_t n, void *stream);
int shmemg_int64_min_reduce(shmemg_team_t team, int64_t *dst, const int64_t *src, uint64_t n, void *stream);
int shmemg_float_sum_reduce(shmemg_team_t team, float *dst, const float *src, uint64_t n, void *stream);
int shmemg_float_max_reduce(shmemg_team_t team, float *dst, const float *src, uint64_t n, void *stream);
int shmemg_float_min_reduce(shmemg_team_t team, float *dst, const float *src, uint64_t n, void *stream);

/* Reduced-precision float payloads (a precision extension of the float sum reduce;
 * not in the paper).  quantize: each member encodes its n floats `src` into codes `q`
 * (bf16: 2 bytes, e4m3: 1 byte each) and per-128-element scales (ceil(n/128) floats):
 * s = max|x| / R (R = 1 for bf16, 448 for e4m3; 1 if the block is all zero),
 * q = RNE-with-saturation(x / s).  qsum_reduce: every member's float dst[k] =
 * compensated (Neumaier) binary32 sum, in team-rank order, of q_r[k] * s_r[k/128]. */
int shmemg_quantize(shmemg_team_t team, void *q, float *scales, const float *src, int fmt,
                    uint64_t n, void *stream);
int shmemg_qsum_reduce(shmemg_team_t team, float *dst, const void *q, const float *scales,
                       int fmt, uint64_t n, void *stream);

/* ----------------------------------------------------------------- scripts */
/* One operation of a scripted stream (64 bytes).  Offsets are symmetric byte offsets
 * inside a partition.  kind: */
enum {
    SHMEMG_OP_PUT = 1, SHMEMG_OP_GET = 2, SHMEMG_OP_PUT_NBI = 3, SHMEMG_OP_GET_NBI = 4,
    SHMEMG_OP_FETCH_ADD = 5, SHMEMG_OP_COMPARE_SWAP = 6, SHMEMG_OP_FETCH_XOR = 7,
    SHMEMG_OP_PUT_SIGNAL = 8, SHMEMG_OP_WAIT_UNTIL = 9,
    SHMEMG_OP_BARRIER_ALL = 10, SHMEMG_OP_QUIET = 11, SHMEMG_OP_FENCE = 12,
    SHMEMG_OP_BROADCAST = 13, SHMEMG_OP_FCOLLECT = 14, SHMEMG_OP_ALLTOALL = 15,
    SHMEMG_OP_REDUCE = 16, SHMEMG_OP_TEAM_SYNC = 17
};
/* Bits 8-15 of `kind` are flags.  SHMEMG_OP_WARP issues the op at warp scope (Sec. 6.3
 * participation scopes): one warp of the issuing PE (put, get, their _nbi forms,
 * put_signal) or of every member PE (collectives, team_sync, barrier_all) performs it,
 * with the same result as the PE-scope form; on other kinds it is invalid. */
#define SHMEMG_OP_KIND_MASK 0xFFu
#define SHMEMG_OP_WARP 0x100u
/* Device contexts (Sec. 6.2): `sub` of put_nbi / get_nbi picks the context, 0 = the
 * default device context, 1..SHMEMG_DEVICE_CTX_COUNT-1 explicit contexts; `sub` of
 * quiet / fence picks the context it completes, or SHMEMG_CTX_ALL.  Each explicit
 * context is an independent completion domain: its non-blocking transfers move in the
 * background and only quiet or fence on that context -- or on all -- waits for them;
 * barriers and collectives quiet the default context only.  Every context is complete
 * when the script ends.  With CTA PEs and no hardware clusters, when the GPU holds two
 * CTAs per PE, shmemg_run_script launches a context agent per PE (a second CTA whose TMA
 * bulk copies run while the PE goes on; set SHMEMG_CTX_AGENTS=0 to turn the agents off);
 * otherwise the PE's own bulk engine advances them at every later op of the PE.  One
 * script runs at a time (concurrent scripts share the agents' mailboxes).
 * Transfers whose addresses or length are not 16-byte multiples (or with the bulk
 * engine off) complete at once, as on the default context. */
#define SHMEMG_DEVICE_CTX_COUNT 4
#define SHMEMG_CTX_ALL 0xFF
typedef struct {
    uint32_t kind;     /* SHMEMG_OP_* | flags */
    uint8_t dtype;     /* AMO / reduce element type */
    uint8_t sub;       /* reduce op, signal op, wait comparison, or context (nbi, quiet, fence) */
    uint16_t team;     /* collectives */
    int32_t pe;        /* target PE (RMA, AMO, signal); root team rank (broadcast) */
    int32_t issuer;    /* issuing PE (RMA, AMO, signal, wait); -1 for collectives */
    uint64_t dst;      /* destination / AMO target / waited signal offset */
    uint64_t src;
    uint64_t n;        /* bytes, or elements for reduce */
    int64_t operand;   /* AMO operand, signal value, wait value */
    int64_t cond;      /* compare_swap condition */
    uint64_t aux;      /* put_signal: signal word offset */
} shmemg_op_t;

/* Device-initiated execution of a script (Sec. 6.3 device-initiated path): one
 * cooperative launch in which every PE (CTA or cluster) walks the list and issues, in
 * list order, the point-to-point ops it is the issuer of and its part of every
 * collective of a team it belongs to.  Collectives and barriers quiet and synchronise
 * their team on entry and exit.  Ops between two synchronising ops run concurrently
 * on different PEs: the script must be race-free there for a deterministic heap.
 * fetched[i] (caller's device array of nops) receives the old value of AMO op i.
 * `ops` is a device array, checked on the device as it is read: an invalid op (a PE or
 * byte range outside the heap, a misaligned AMO target, a destroyed team) ends the
 * script at that op and records SHMEMG_ERR_INVALID_ARG with the op's index in the
 * status word; the ops before it have run.  Needs every PE co-resident:
 * SHMEMG_ERR_UNSUPPORTED if the GPU cannot hold them. */
int shmemg_run_script(const shmemg_op_t *ops, int64_t nops, int64_t *fetched, void *stream);
/* The plain launch-per-op path: the same list, from HOST memory, executed in list
 * order by one stream-triggered host call per op on `stream`. */
int shmemg_run_script_host(const shmemg_op_t *ops, int64_t nops, int64_t *fetched, void *stream);

/* ----------------------------------------------------------------- AMO stress */
/* Device-initiated AMO stream over an int64 table distributed across all PEs: word w
 * lives on PE w / words_per_pe at symmetric offset table + (w % words_per_pe) * 8.
 * One CTA per PE; PE p issues ops [p*nops/npes, (p+1)*nops/npes) in order.  Op i
 * (packed uint32: bits 0..26 word, bits 27..28 code 0 fetch_add, 1 compare_swap,
 * 2 fetch_xor) takes r = splitmix64 counter draw (op_seed ^ i): fetch_add adds
 * (r mod 2^20) + 1, compare_swap swaps in r if the word equals its initial value
 * splitmix64(table_seed ^ w), fetch_xor xors r (1 if r is 0).  fetched[i] (device, may
 * be NULL) gets the old value.  flags bit 0: warp-aggregate fetch_add/fetch_xor on
 * equal targets (the aggregated ops are consecutive in the serial order).  flags bit 1
 * (takes precedence): combine the ops of each CTA tile of 1024 that have the same word
 * and code -- fetch_add, fetch_xor and compare_swap -- into one atomic per group (again
 * consecutive in the serial order; a compare_swap whose swap value equals the compare
 * value is applied on its own).  An op whose
 * word is >= npes*words_per_pe (or whose code is 3) is skipped and recorded in the
 * status word (SHMEMG_ERR_INVALID_ARG, detail = op index). */
#define SHMEMG_AMO_AGGREGATE 1u
#define SHMEMG_AMO_COMBINE_BLOCK 2u
int shmemg_amo_stream(int64_t *table, uint64_t words_per_pe, const uint32_t *ops, uint64_t nops,
                      uint64_t op_seed, uint64_t table_seed, int64_t *fetched, uint32_t flags,
                      void *stream);

/* Put-with-signal ping-pong between PE pairs (2k, 2k+1), one CTA per PE, cooperative
 * launch: for t in 0..iters-1 PE 2k puts `payload` bytes of its `buf` into the peer's
 * `buf` + payload and adds 1 to the peer's signal `sig`, then waits for its own signal
 * to reach t+1; PE 2k+1 answers in kind.  lat_ns[k*iters + t] (device, npairs*iters
 * uint64, may be NULL) receives round trip t of pair k in ns (globaltimer).  buf must
 * hold 2*payload bytes per PE; sig one uint64 per PE, zero before the call.  Needs
 * pe_mode CTA and 2*npairs co-resident CTAs (else SHMEMG_ERR_UNSUPPORTED). */
int shmemg_pingpong(void *buf, uint64_t *sig, uint64_t payload, int npairs, int iters,
                    uint64_t *lat_ns, void *stream);

/* The ping-pong of shmemg_pingpong between the two CTAs of each pair inside one
 * thread-block cluster, through distributed shared memory (Sec. 4.2 direct pointers,
 * Sec. 6.3 device shared team): the payload goes into the peer's shared-memory window
 * and the signal is a word of that window (cluster-scope release add, acquire poll).
 * At the end PE p writes the last payload it received to its buf + payload and adds
 * the rounds it received to its `sig`: the heap ends exactly as after shmemg_pingpong.
 * Needs pe_mode CTA with cluster_dim >= 2 (each pair inside one device shared team) and
 * 2*npairs a multiple of cluster_dim (else SHMEMG_ERR_UNSUPPORTED), payload <=
 * SHMEMG_PINGPONG_CLUSTER_MAX; other arguments as shmemg_pingpong.  A pair's CTAs share
 * a cluster, which the hardware schedules at once, so no cooperative launch is needed.
 * Launched without its clusters (by a profiler's replay, say) the kernel records
 * SHMEMG_ERR_UNSUPPORTED in the status word and touches nothing. */
#define SHMEMG_PINGPONG_CLUSTER_MAX (64u << 10)
int shmemg_pingpong_cluster(void *buf, uint64_t *sig, uint64_t payload, int npairs, int iters,
                            uint64_t *lat_ns, void *stream);

/* ----------------------------------------------------------------- halo exchange */
/* A GPU-resident halo exchange in a stencil code (Sec. 4.4, case study 1): the npes PEs
 * form a px x py grid (PE = y*px + x) over a periodic 2-D grid of binary32 values; PE p
 * owns an nx x ny tile (row-major, nx a multiple of 4) and runs `iters` Jacobi sweeps
 * out = 0.25 * ((up + down) + (left + right)) (RNE, in this order).  Symmetric objects:
 *   tiles  2*nx*ny floats: tile 0 holds the input; after the call the result is in tile
 *          (iters & 1);
 *   halos  2*hs floats, hs = shmemg_halo_stride(nx, ny) = 2*nx + 2*ny4 with ny4 = ny
 *          rounded up to a multiple of 4 (work space: north and south rows, west and
 *          east columns, each part 16-byte aligned);
 *   sigs   4 uint64, zero before the call (left zero after a successful call).
 * shmemg_halo_jacobi: one cooperative launch; after each sweep a PE stores its new
 * boundary rows and columns straight into its four neighbours' halo buffers (device-
 * initiated puts fused into the sweep), then signals each neighbour (put-with-signal,
 * Sec. 7); before each sweep it waits for its four signals (bounded wait_until).
 * shmemg_halo_jacobi_plain: the same sweeps, one stream-ordered launch per sweep (the
 * plain launch-per-op path: kernel boundaries replace the signals).  tiles and halos
 * 16-byte aligned, px*py == npes, else SHMEMG_ERR_INVALID_ARG. */
uint64_t shmemg_halo_stride(int nx, int ny);
int shmemg_halo_jacobi(float *tiles, float *halos, uint64_t *sigs, int px, int py, int nx, int ny,
                       int iters, void *stream);
int shmemg_halo_jacobi_plain(float *tiles, float *halos, uint64_t *sigs, int px, int py, int nx,
                             int ny, int iters, void *stream);

/* ----------------------------------------------------------------- batched collectives */
/* Many teams' uneven collectives in one persistent launch captured in a CUDA graph. */
typedef struct {
    int32_t start;      /* first world PE of the team; members start .. start+size-1 */
    int32_t size;
    int32_t dtype;      /* SHMEMG_FLOAT (tree sum), SHMEMG_INT64 (exact sum), or
                           SHMEMG_FLOAT with fmt >= 0 (quantised payload sum) */
    int32_t fmt;        /* -1, or SHMEMG_FMT_BF16 / _E4M3 for quantised payloads */
    uint64_t n;         /* elements per PE */
    void *dst;          /* symmetric: float / int64 output, n elements */
    const void *src;    /* symmetric: float / int64 input, or quantised codes */
    const float *scales; /* symmetric scales for quantised payloads, else NULL */
} shmemg_coll_desc_t;
typedef struct {
    int32_t tile_elems;   /* elements per work item; 0 = autotune */
    int32_t ctas_per_sm;  /* 0 = occupancy maximum */
    int32_t threads;      /* threads per CTA, 0 = 256 */
    int32_t deep;         /* 0: the kernel held to 3 CTAs per SM; 1: the one held to 2 CTAs
                             per SM whose quantised sums load 16 members ahead, not 8 */
} shmemg_tune_t;
typedef struct shmemg_batch_s *shmemg_batch_t;
/* Validates and uploads the descriptors, plans work items largest-first and captures
 * one persistent launch in a CUDA graph.  `tune` may be NULL (defaults). */
int shmemg_batch_create(const shmemg_coll_desc_t *descs, int count, const shmemg_tune_t *tune,
                        shmemg_batch_t *out);
int shmemg_batch_launch(shmemg_batch_t batch, void *stream);
/* Times each candidate plan with CUDA events on `stream`, keeps the fastest, re-captures
 * the graph, and reports the choice in *chosen (may be NULL). */
int shmemg_batch_autotune(shmemg_batch_t batch, void *stream, shmemg_tune_t *chosen);
int shmemg_batch_destroy(shmemg_batch_t batch);

/* Allocation-free batched sum reduce.  The paper has no counterpart: this is a
 * service of this library for callers that cannot allocate device memory -- a host
 * framework whose caching allocator already holds the GPU's memory, or a
 * latency-critical loop that must not call cudaMalloc/cudaFree (cudaFree synchronises
 * the whole device).  It computes exactly what shmemg_batch_create + shmemg_batch_launch
 * compute for the same descriptors and tile size (largest-first work items, one launch
 * of the same kernel on `stream`), but keeps the team table, the work items and the two
 * work counters in one array compiled into the library (about 560 KiB, held by every GPU
 * that loads the library until the process exits) instead of allocating them.  The
 * caller still passes the inputs and outputs (symmetric objects in the descriptors).
 * Limits: at most SHMEMG_NOALLOC_MAX_TEAMS descriptors and SHMEMG_NOALLOC_MAX_ITEMS work
 * items (sum over teams of ceil(n / tile)); larger requests return
 * SHMEMG_ERR_INVALID_ARG and launch nothing.  tile_elems: a multiple of 128, 0 = 16384.
 * The first call on a device looks the array's device address up (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Every
 * call overwrites the array (the counters are cleared on `stream` before the launch):
 * calls whose work overlaps on the GPU -- on different streams, or on different host
 * threads -- race on it and give wrong results; order them (one stream, or events). */
#define SHMEMG_NOALLOC_MAX_TEAMS 1024
#define SHMEMG_NOALLOC_MAX_ITEMS 65536
int shmemg_batch_reduce_noalloc(const shmemg_coll_desc_t *descs, int count, int tile_elems, void *stream);

/* ----------------------------------------------------------------- serving */
/* A persistent, device-resident progress kernel (paper Sec. 3 and 7: persistent
 * kernels; the paper leaves their progress guarantee to the implementation, this one
 * documents it below).  CTA 0 admits: it acquire-polls a request ring in mapped host
 * memory, gives each request a slot and its destination pages (the same page range on
 * every PE the request writes, first fit in per-PE page bitmaps), and publishes it to a
 * device work queue.  The other CTAs take (request, tile) work items from the head of
 * that queue, so requests admitted while others run share the GPU tile by tile
 * (continuous batching).  The CTA that finishes a request's last tile writes its
 * completion record to mapped host memory and frees its pages and slot.
 *
 * Request kinds (SHMEMG_OP_*):
 *   PUT      n bytes of `src` on `issuer` -> fresh pages on `pe`
 *   GET      n bytes of `src` on `pe`     -> fresh pages on `issuer`
 *   FETCH_ADD / COMPARE_SWAP / FETCH_XOR  int64 on table word `word` (word w lives on
 *            PE w / amo_words at amo_offset + 8*(w % amo_words)); operand, cond
 *   REDUCE   sum all-reduce over PEs pe .. pe+issuer-1 of n elements at `src`
 *            (dtype SHMEMG_FLOAT with fmt 0xFF: fp32 by the rank-pairwise tree; dtype
 *            SHMEMG_FLOAT with fmt SHMEMG_FMT_BF16: bf16 codes at src, per-128 scales at
 *            symmetric offset `cond`, Neumaier fp32 accumulation; dtype SHMEMG_INT64:
 *            exact) into fresh pages on every member
 *   ALLTOALL blocks of n bytes over PEs pe .. pe+issuer-1 from `src` into fresh pages
 * Offsets `src` (and `cond` for bf16 scales) are symmetric byte offsets of caller data
 * the server only reads: 16-byte aligned; n a multiple of 8 (RMA), 4 (REDUCE) or 16
 * (ALLTOALL).
 *
 * Staged payloads (flags & SHMEMG_REQ_STAGED; not for AMOs).  The request brings its
 * input instead of naming caller data: `word` is the payload's seed, `src` and `cond`
 * are ignored.  Admission takes one page range, the request's region, on every PE the
 * request touches (PUT/GET: the source and the destination PE; REDUCE/ALLTOALL: every
 * member), laid out from its start R (16-byte aligned parts):
 *   PUT/GET    [R, R + a) destination, [R + a, R + 2a) source, a = n rounded up to 16
 *   REDUCE     fp32 and int64: [R, R + n*e) source and destination (in place);
 *              bf16: [R, R + c4) fp32 destination, then the source: codes at R + c4
 *              (2n bytes) and scales at R + c4 + c2 (4*ceil(n/128) bytes), where c4, c2
 *              are 4n and 2n rounded up to 16
 *   ALLTOALL   [R, R + P*n) destination blocks, [R + P*n, R + 2*P*n) source blocks
 * The request first writes its source on every source PE p: 32-bit word j of the source
 * part (at byte 4j from its start) is
 *   w(j) = (b((z >> (56 - 16q)) & 255) << 16) | b((z >> (48 - 16q)) & 255),  q = j mod 4,
 * where z is the first output of Steele, Lea and Flood's SplitMix64 stream started at
 * state seed ^ ((p << 40) | floor(j / 4)) -- one draw gives four words, two of its bytes
 * each, high bytes first -- and b(k) = ((k & 128) << 8) | 0x3F80 | (k & 127), the
 * bfloat16 code of (-1)^(k >> 7) * (1 + (k & 127) / 128); then it runs the operation on
 * that source like any other request.
 *
 * The result is the fetched value (AMO) or a checksum of the output:
 * sum over its little-endian 32-bit words w_i (members' outputs concatenated in team
 * rank order) of w_i * (2i + 1), modulo 2^64.  Invalid requests complete with an error
 * status.  Progress: the kernel needs no host action to progress; it exits on stop,
 * after idle_ns without requests, or after max_ns in total. */
#define SHMEMG_REQ_STAGED 1u   /* shmemg_req_t.flags: the request stages its own payload */
typedef struct {
    uint32_t kind;
    uint8_t dtype;
    uint8_t fmt;
    uint16_t flags;     /* SHMEMG_REQ_STAGED or 0 */
    int32_t pe;
    int32_t issuer;     /* RMA/AMO issuing PE; REDUCE/ALLTOALL team size */
    uint64_t n;
    uint64_t word;      /* AMO: table word; staged payload: its seed */
    int64_t operand;
    int64_t cond;
    uint64_t src;       /* symmetric offset of the request's input */
    uint64_t ticket;    /* set by submit */
} shmemg_req_t;
typedef struct {
    uint64_t ticket;
    uint64_t t_admit_ns;   /* globaltimer when the request was admitted (or its kernel began) */
    uint64_t t_done_ns;    /* globaltimer at completion */
    uint64_t result;       /* AMO: fetched value; others: checksum of the output */
    int32_t status;        /* SHMEMG_SUCCESS or an error */
    uint32_t seq;          /* record sequence number + 1, written last */
} shmemg_completion_t;
typedef struct {
    int32_t workers;          /* worker CTAs (0 = every CTA the GPU holds at once, minus one) */
    int32_t ring_slots;       /* request / completion ring capacity (power of two, 0 = 65536) */
    int32_t max_inflight;     /* admitted-but-unfinished request limit (0 = 1024) */
    int32_t reserved0;
    uint64_t page_bytes;      /* admission page size (multiple of 256, 0 = 65536) */
    uint64_t arena_offset;    /* symmetric offset of the pageable arena (destinations) */
    uint64_t arena_bytes;     /* per-PE bytes of the arena (<= 4096 pages) */
    uint64_t amo_offset;      /* symmetric offset of the AMO table */
    uint64_t amo_words;       /* AMO table words per PE */
    uint64_t idle_ns;         /* exit after this long without a request (0 = 60 s) */
    uint64_t max_ns;          /* exit after this long in total (0 = 600 s) */
} shmemg_server_cfg_t;
typedef struct shmemg_server_s *shmemg_server_t;
/* Launches the progress kernel (a cooperative launch; it occupies `stream` until it
 * exits, so give it a stream of its own).  Allocates the server's device queues and
 * mapped host rings. */
int shmemg_server_start(const shmemg_server_cfg_t *cfg, void *stream, shmemg_server_t *out);
/* Publishes one request (release store of the ring tail to device-visible memory);
 * SHMEMG_ERR_BUSY if the ring is full.  *ticket (may be NULL) gets its ticket. */
int shmemg_server_submit(shmemg_server_t s, const shmemg_req_t *req, uint64_t *ticket);
/* Submits reqs[i] at host time t0 + arrival_ns[i] (CLOCK_MONOTONIC; spins, retries while
 * the ring is full); *t0_ns receives t0.  A native feeder for open-loop arrivals. */
int shmemg_server_feed(shmemg_server_t s, const shmemg_req_t *reqs, int count, const uint64_t *arrival_ns,
                       uint64_t *t0_ns);
/* Copies up to `max` new completion records in completion order; *got = how many. */
int shmemg_server_poll(shmemg_server_t s, shmemg_completion_t *out, int max, int *got);
/* Sets the stop flag and waits (bounded by 60 s) for the kernel to drain and exit;
 * frees the server.  SHMEMG_ERR_TIMEOUT if it did not exit in time. */
int shmemg_server_stop(shmemg_server_t s);

/* The plain launch-per-op path for the same requests: one full-grid kernel per request
 * on `stream`, destinations at cfg->arena_offset (requests on one stream never
 * overlap), completion record written to `rec` (host-mapped or device memory). */
int shmemg_request_run(const shmemg_req_t *req, const shmemg_server_cfg_t *cfg, shmemg_completion_t *rec,
                       void *stream);
/* Launches reqs[i] at host time t0 + arrival_ns[i] (CLOCK_MONOTONIC), one kernel each on
 * `stream`; recs (count records, host-mapped) receive the completions; *t0_ns gets t0. */
int shmemg_plain_feed(const shmemg_req_t *reqs, int count, const uint64_t *arrival_ns,
                      const shmemg_server_cfg_t *cfg, shmemg_completion_t *recs, void *stream, uint64_t *t0_ns);
/* globaltimer value now (ns), read by a tiny kernel. */
int shmemg_device_time_ns(uint64_t *out);
/* Offset between the device globaltimer and the host CLOCK_MONOTONIC (device - host,
 * ns), from the tightest of `rounds` launch round trips; *err_ns = half that round trip. */
int shmemg_clock_offset(int rounds, int64_t *offset_ns, uint64_t *err_ns);

#ifdef __cplusplus
}
#endif
#endif /* SHMEMG_H */
