"""Python binding of libshmemg (ctypes): argument marshalling only.

Every operation runs in the library's CUDA kernels; there is no Python or CPU
implementation of any of them.  If the shared library is missing, importing a
function raises immediately.  PyTorch provides the device memory of the symmetric
heap and the streams.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import builder as _build

_lib = None

# status codes / enums (mirror include/shmemg.h)
SUCCESS = 0
ERR_INVALID_ARG, ERR_NOT_INITIALIZED, ERR_OUT_OF_HEAP, ERR_NOT_SYMMETRIC = -1, -2, -3, -4
ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_CUDA, ERR_BUSY, ERR_DEVICE = -5, -6, -7, -8, -9
PE_MODE_CTA, PE_MODE_CLUSTER = 0, 1
INT32, INT64, FLOAT, UINT64 = 0, 1, 2, 3
SUM, MAX, MIN = 0, 1, 2
SIGNAL_SET, SIGNAL_ADD = 0, 1
CMP_EQ, CMP_NE, CMP_GT, CMP_GE, CMP_LT, CMP_LE = range(6)
FMT_BF16, FMT_E4M3 = 0, 1
TEAM_WORLD, TEAM_SHARED = 0, 1
RESERVED_BYTES = 4 << 20
AMO_AGGREGATE = 1
AMO_COMBINE_BLOCK = 2

CAP_NAMES = ["GPU_AWARE_HOST", "DEVICE_RMA", "DEVICE_AMO", "DEVICE_SIGNAL", "DEVICE_COLL", "STREAM_ORDERED",
             "DEVICE_CTX_DEFAULT", "EXPLICIT_DEVICE_CTX", "DEVICE_TEAMS", "PTR_DEVICE", "PTR_HOST",
             "PROGRESS_GPU", "HOST_PROGRESS_REQUIRED", "MIXED_HOST_DEVICE_COLL", "PERSISTENT_SERVER",
             "BATCHED_COLL", "QUANTIZED_REDUCE"]


class ShmemgError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = lib().shmemg_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})")


class InitAttr(C.Structure):
    _fields_ = [("npes", C.c_int32), ("pe_mode", C.c_int32), ("cluster_dim", C.c_int32), ("reserved0", C.c_int32),
                ("heap_bytes_per_pe", C.c_uint64), ("heap_ptr", C.c_void_p), ("heap_bytes", C.c_uint64),
                ("stream", C.c_void_p), ("wait_timeout_ns", C.c_uint64)]


class DeviceCtx(C.Structure):
    _fields_ = [("heap", C.c_void_p), ("pe_stride", C.c_uint64), ("npes", C.c_int32), ("pe_mode", C.c_int32),
                ("cluster_dim", C.c_int32), ("reserved0", C.c_int32), ("state", C.c_void_p),
                ("timeout_ns", C.c_uint64)]


class Caps(C.Structure):
    _fields_ = [("flags", C.c_uint64), ("default_heap", C.c_int32), ("path", C.c_int32), ("rma_scopes", C.c_uint32),
                ("coll_scopes", C.c_uint32), ("device_ordinal", C.c_int32), ("pe_mode", C.c_int32),
                ("cluster_dim", C.c_int32), ("team_n_pes", C.c_int32), ("shared_team_size", C.c_int32),
                ("device_ctx_count", C.c_int32), ("heap_bytes_per_pe", C.c_uint64), ("heap_free_bytes", C.c_uint64),
                ("wait_timeout_ns", C.c_uint64)]


class CollDesc(C.Structure):
    _fields_ = [("start", C.c_int32), ("size", C.c_int32), ("dtype", C.c_int32), ("fmt", C.c_int32),
                ("n", C.c_uint64), ("dst", C.c_void_p), ("src", C.c_void_p), ("scales", C.c_void_p)]


class Tune(C.Structure):
    _fields_ = [("tile_elems", C.c_int32), ("ctas_per_sm", C.c_int32), ("threads", C.c_int32),
                ("deep", C.c_int32)]


class Req(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("dtype", C.c_uint8), ("fmt", C.c_uint8), ("flags", C.c_uint16),
                ("pe", C.c_int32), ("issuer", C.c_int32), ("n", C.c_uint64), ("word", C.c_uint64),
                ("operand", C.c_int64), ("cond", C.c_int64), ("src", C.c_uint64), ("ticket", C.c_uint64)]


REQ_DTYPE = np.dtype([("kind", "<u4"), ("dtype", "u1"), ("fmt", "u1"), ("flags", "<u2"), ("pe", "<i4"),
                      ("issuer", "<i4"), ("n", "<u8"), ("word", "<u8"), ("operand", "<i8"), ("cond", "<i8"),
                      ("src", "<u8"), ("ticket", "<u8")])
COMPLETION_DTYPE = np.dtype([("ticket", "<u8"), ("t_admit_ns", "<u8"), ("t_done_ns", "<u8"), ("result", "<u8"),
                             ("status", "<i4"), ("seq", "<u4")])
FMT_F32 = 0xFF


class Completion(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("t_admit_ns", C.c_uint64), ("t_done_ns", C.c_uint64),
                ("result", C.c_uint64), ("status", C.c_int32), ("seq", C.c_uint32)]


class ServerCfg(C.Structure):
    _fields_ = [("workers", C.c_int32), ("ring_slots", C.c_int32), ("max_inflight", C.c_int32),
                ("reserved0", C.c_int32), ("page_bytes", C.c_uint64), ("arena_offset", C.c_uint64),
                ("arena_bytes", C.c_uint64), ("amo_offset", C.c_uint64), ("amo_words", C.c_uint64),
                ("idle_ns", C.c_uint64), ("max_ns", C.c_uint64)]


P, I, U64, I64, U32 = C.c_void_p, C.c_int, C.c_uint64, C.c_int64, C.c_uint32
_SIGS = {
    "shmemg_required_heap_bytes": [I, U64, P],
    "shmemg_init": [P],
    "shmemg_finalize": [],
    "shmemg_initialized": [P],
    "shmemg_n_pes": [P],
    "shmemg_device_ctx": [P],
    "shmemg_malloc": [U64, P],
    "shmemg_calloc": [U64, P, P],
    "shmemg_free": [P],
    "shmemg_ptr": [P, I, P],
    "shmemg_team_split_strided": [I, I, I, I, P],
    "shmemg_team_destroy": [I],
    "shmemg_team_n_pes": [I, P],
    "shmemg_team_translate_pe": [I, I, I, P],
    "shmemg_query_capabilities": [I, P],
    "shmemg_get_status": [P, P],
    "shmemg_clear_status": [P],
    "shmemg_putmem": [P, P, U64, I, I, P],
    "shmemg_putmem_nbi": [P, P, U64, I, I, P],
    "shmemg_getmem": [P, P, U64, I, I, P],
    "shmemg_getmem_nbi": [P, P, U64, I, I, P],
    "shmemg_int64_atomic_fetch_add": [P, I64, I, P, P],
    "shmemg_int64_atomic_compare_swap": [P, I64, I64, I, P, P],
    "shmemg_int64_atomic_fetch_xor": [P, I64, I, P, P],
    "shmemg_int32_atomic_fetch_add": [P, C.c_int32, I, P, P],
    "shmemg_int32_atomic_compare_swap": [P, C.c_int32, C.c_int32, I, P, P],
    "shmemg_int32_atomic_fetch_xor": [P, C.c_int32, I, P, P],
    "shmemg_putmem_signal": [P, P, U64, P, U64, I, I, I, P],
    "shmemg_signal_wait_until": [P, I, I, U64, P],
    "shmemg_fence": [P],
    "shmemg_quiet": [P],
    "shmemg_barrier_all": [P],
    "shmemg_team_sync": [I, P],
    "shmemg_broadcastmem": [I, P, P, U64, I, P],
    "shmemg_fcollectmem": [I, P, P, U64, P],
    "shmemg_alltoallmem": [I, P, P, U64, P],
    "shmemg_reduce": [I, P, P, U64, I, I, P],
    "shmemg_quantize": [I, P, P, P, I, U64, P],
    "shmemg_qsum_reduce": [I, P, P, P, I, U64, P],
    "shmemg_run_script": [P, I64, P, P],
    "shmemg_run_script_host": [P, I64, P, P],
    "shmemg_amo_stream": [P, U64, P, U64, U64, U64, P, U32, P],
    "shmemg_pingpong": [P, P, U64, I, I, P, P],
    "shmemg_pingpong_cluster": [P, P, U64, I, I, P, P],
    "shmemg_halo_jacobi": [P, P, P, I, I, I, I, I, P],
    "shmemg_halo_jacobi_plain": [P, P, P, I, I, I, I, I, P],
    "shmemg_batch_create": [P, I, P, P],
    "shmemg_batch_launch": [P, P],
    "shmemg_batch_autotune": [P, P, P],
    "shmemg_batch_destroy": [P],
    "shmemg_batch_reduce_noalloc": [P, I, I, P],
    "shmemg_server_start": [P, P, P],
    "shmemg_server_submit": [P, P, P],
    "shmemg_server_poll": [P, P, I, P],
    "shmemg_server_stop": [P],
    "shmemg_server_feed": [P, P, I, P, P],
    "shmemg_request_run": [P, P, P, P],
    "shmemg_plain_feed": [P, I, P, P, P, P, P],
    "shmemg_clock_offset": [I, P, P],
    "shmemg_device_time_ns": [P],
}
for _dt in ("int32", "int64", "float"):
    for _op in ("sum", "max", "min"):
        _SIGS[f"shmemg_{_dt}_{_op}_reduce"] = [I, P, P, U64, P]


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded libshmemg; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libshmemg is not built ({path} missing); run paper_2607_08006_gb300.build.build()")
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = C.c_int
        L.shmemg_strerror.argtypes = [I]
        L.shmemg_strerror.restype = C.c_char_p
        L.shmemg_halo_stride.argtypes = [I, I]
        L.shmemg_halo_stride.restype = C.c_uint64
        _lib = L
    return _lib


def _call(name, *args):
    f = getattr(lib(), name, None)
    if f is None:
        raise RuntimeError(f"{name} is not exported by libshmemg")
    rc = f(*args)
    if rc != SUCCESS:
        raise ShmemgError(rc, name)
    return rc


def _stream(s):
    """torch.cuda.Stream / int / None -> cudaStream_t as int."""
    if s is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "ptr"):
        return x.ptr
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer of {type(x)}")


@dataclass
class Sym:
    """A symmetric object: canonical pointer (PE 0's copy) and byte offset."""
    ptr: int
    offset: int
    nbytes: int


class Heap:
    """The symmetric heap: one torch uint8 device tensor carved into npes partitions."""

    def __init__(self, npes, heap_bytes_per_pe, pe_mode=PE_MODE_CTA, cluster_dim=1, timeout_ns=0, stream=None):
        import torch

        need = C.c_uint64(0)
        _call("shmemg_required_heap_bytes", npes, heap_bytes_per_pe, C.byref(need))
        self.tensor = torch.empty(need.value, dtype=torch.uint8, device="cuda")
        self.npes, self.H = npes, heap_bytes_per_pe
        a = InitAttr(npes=npes, pe_mode=pe_mode, cluster_dim=cluster_dim, heap_bytes_per_pe=heap_bytes_per_pe,
                     heap_ptr=self.tensor.data_ptr(), heap_bytes=need.value, stream=_stream(stream),
                     wait_timeout_ns=timeout_ns)
        _call("shmemg_init", C.byref(a))
        self.base = self.tensor.data_ptr() + RESERVED_BYTES
        self.live = True

    def close(self):
        if self.live:
            _call("shmemg_finalize")
            self.live = False

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # memory ----------------------------------------------------------------------
    def malloc(self, nbytes) -> Sym:
        p = C.c_void_p(0)
        _call("shmemg_malloc", nbytes, C.byref(p))
        return Sym(p.value, p.value - self.base, nbytes)

    def calloc(self, nbytes, stream=None) -> Sym:
        p = C.c_void_p(0)
        _call("shmemg_calloc", nbytes, C.byref(p), _stream(stream))
        return Sym(p.value, p.value - self.base, nbytes)

    def free(self, sym: Sym):
        _call("shmemg_free", sym.ptr)

    def sym(self, offset: int, nbytes: int = 0) -> Sym:
        return Sym(self.base + offset, offset, nbytes)

    def partitions(self):
        """[npes, H] uint8 view of the partitions (device)."""
        return self.tensor[RESERVED_BYTES:RESERVED_BYTES + self.npes * self.H].view(self.npes, self.H)

    def view(self, sym, pe, dtype, count=None):
        """torch view of PE pe's copy of a symmetric object."""
        import torch

        off = sym.offset if isinstance(sym, Sym) else int(sym)
        es = torch.empty((), dtype=dtype).element_size()
        if count is None:
            count = sym.nbytes // es
        start = RESERVED_BYTES + pe * self.H + off
        return self.tensor[start:start + count * es].view(dtype)

    def ptr(self, sym, pe) -> int:
        out = C.c_void_p(0)
        _call("shmemg_ptr", _ptr(sym), pe, C.byref(out))
        return out.value


def required_heap_bytes(npes, H):
    out = C.c_uint64(0)
    _call("shmemg_required_heap_bytes", npes, H, C.byref(out))
    return out.value


def n_pes():
    v = C.c_int(0)
    _call("shmemg_n_pes", C.byref(v))
    return v.value


def device_ctx() -> DeviceCtx:
    c = DeviceCtx()
    _call("shmemg_device_ctx", C.byref(c))
    return c


def query_capabilities(team=TEAM_WORLD) -> dict:
    c = Caps()
    _call("shmemg_query_capabilities", team, C.byref(c))
    d = {f: getattr(c, f) for f, _ in Caps._fields_ if not f.startswith("reserved")}
    d["flag_names"] = [n for i, n in enumerate(CAP_NAMES) if c.flags >> i & 1]
    return d


def get_status():
    code, detail = C.c_int(0), C.c_int64(0)
    _call("shmemg_get_status", C.byref(code), C.byref(detail))
    return code.value, detail.value


def clear_status(stream=None):
    _call("shmemg_clear_status", _stream(stream))


def strerror(code) -> str:
    return lib().shmemg_strerror(code).decode()


# teams -----------------------------------------------------------------------------
def team_split_strided(parent, start, stride, size) -> int:
    t = C.c_int(0)
    _call("shmemg_team_split_strided", parent, start, stride, size, C.byref(t))
    return t.value


def team_destroy(team):
    _call("shmemg_team_destroy", team)


def team_n_pes(team) -> int:
    v = C.c_int(0)
    _call("shmemg_team_n_pes", team, C.byref(v))
    return v.value


def team_translate_pe(src_team, src_pe, dest_team) -> int:
    v = C.c_int(0)
    _call("shmemg_team_translate_pe", src_team, src_pe, dest_team, C.byref(v))
    return v.value


# RMA / AMO / signal ----------------------------------------------------------------
def putmem(dst, src, n, pe, issuer, stream=None, nbi=False):
    _call("shmemg_putmem_nbi" if nbi else "shmemg_putmem", _ptr(dst), _ptr(src), n, pe, issuer, _stream(stream))


def getmem(dst, src, n, pe, issuer, stream=None, nbi=False):
    _call("shmemg_getmem_nbi" if nbi else "shmemg_getmem", _ptr(dst), _ptr(src), n, pe, issuer, _stream(stream))


def atomic(kind, dtype, target, value, pe, fetched=None, cond=0, stream=None):
    """kind: 'fetch_add' | 'compare_swap' | 'fetch_xor'; dtype INT32 | INT64."""
    pre = "shmemg_int64_atomic_" if dtype == INT64 else "shmemg_int32_atomic_"
    if kind == "compare_swap":
        _call(pre + kind, _ptr(target), cond, value, pe, _ptr(fetched), _stream(stream))
    else:
        _call(pre + kind, _ptr(target), value, pe, _ptr(fetched), _stream(stream))


def putmem_signal(dst, src, n, sig, sigval, sig_op, pe, issuer, stream=None):
    _call("shmemg_putmem_signal", _ptr(dst), _ptr(src), n, _ptr(sig), sigval, sig_op, pe, issuer, _stream(stream))


def signal_wait_until(sig, pe, cmp, value, stream=None):
    _call("shmemg_signal_wait_until", _ptr(sig), pe, cmp, value, _stream(stream))


def fence(stream=None):
    _call("shmemg_fence", _stream(stream))


def quiet(stream=None):
    _call("shmemg_quiet", _stream(stream))


def barrier_all(stream=None):
    _call("shmemg_barrier_all", _stream(stream))


def team_sync(team, stream=None):
    _call("shmemg_team_sync", team, _stream(stream))


# collectives -----------------------------------------------------------------------
def broadcastmem(team, dst, src, n, root, stream=None):
    _call("shmemg_broadcastmem", team, _ptr(dst), _ptr(src), n, root, _stream(stream))


def fcollectmem(team, dst, src, n, stream=None):
    _call("shmemg_fcollectmem", team, _ptr(dst), _ptr(src), n, _stream(stream))


def alltoallmem(team, dst, src, n, stream=None):
    _call("shmemg_alltoallmem", team, _ptr(dst), _ptr(src), n, _stream(stream))


def reduce(team, dst, src, nelems, dtype, op, stream=None):
    _call("shmemg_reduce", team, _ptr(dst), _ptr(src), nelems, dtype, op, _stream(stream))


def named_reduce(dtype_name, op_name, team, dst, src, nelems, stream=None):
    _call(f"shmemg_{dtype_name}_{op_name}_reduce", team, _ptr(dst), _ptr(src), nelems, _stream(stream))


def quantize(team, q, scales, src, fmt, n, stream=None):
    _call("shmemg_quantize", team, _ptr(q), _ptr(scales), _ptr(src), fmt, n, _stream(stream))


def qsum_reduce(team, dst, q, scales, fmt, n, stream=None):
    _call("shmemg_qsum_reduce", team, _ptr(dst), _ptr(q), _ptr(scales), fmt, n, _stream(stream))


# scripts ---------------------------------------------------------------------------
def run_script(ops_dev, nops, fetched_dev, stream=None):
    """Device-initiated execution of a script held in device memory."""
    _call("shmemg_run_script", _ptr(ops_dev), nops, _ptr(fetched_dev), _stream(stream))


def run_script_host(ops: np.ndarray, fetched_dev, stream=None):
    """Launch-per-op execution of a script held in host memory (numpy records)."""
    ops = np.ascontiguousarray(ops)
    assert ops.dtype.itemsize == 64
    _call("shmemg_run_script_host", ops.ctypes.data_as(C.c_void_p), len(ops), _ptr(fetched_dev), _stream(stream))


# AMO stress / ping-pong --------------------------------------------------------------
def amo_stream(table, words_per_pe, ops_dev, nops, op_seed, table_seed, fetched_dev=None, flags=0, stream=None):
    _call("shmemg_amo_stream", _ptr(table), words_per_pe, _ptr(ops_dev), nops, op_seed, table_seed,
          _ptr(fetched_dev), flags, _stream(stream))


def pingpong(buf, sig, payload, npairs, iters, lat_dev, stream=None):
    _call("shmemg_pingpong", _ptr(buf), _ptr(sig), payload, npairs, iters, _ptr(lat_dev), _stream(stream))


def pingpong_cluster(buf, sig, payload, npairs, iters, lat_dev, stream=None):
    _call("shmemg_pingpong_cluster", _ptr(buf), _ptr(sig), payload, npairs, iters, _ptr(lat_dev), _stream(stream))


def halo_stride(nx, ny):
    """Floats per halo buffer of the halo exchange (2nx + 2 * ny rounded up to 4)."""
    return int(lib().shmemg_halo_stride(nx, ny))


def halo_jacobi(tiles, halos, sigs, px, py, nx, ny, iters, stream=None, plain=False):
    _call("shmemg_halo_jacobi_plain" if plain else "shmemg_halo_jacobi", _ptr(tiles), _ptr(halos), _ptr(sigs),
          px, py, nx, ny, iters, _stream(stream))


# batched collectives -----------------------------------------------------------------
class Batch:
    def __init__(self, descs, tune=None):
        arr = (CollDesc * len(descs))(*descs)
        self._descs = arr
        h = C.c_void_p(0)
        _call("shmemg_batch_create", C.cast(arr, C.c_void_p), len(descs),
              C.byref(tune) if tune is not None else None, C.byref(h))
        self.h = h

    def launch(self, stream=None):
        _call("shmemg_batch_launch", self.h, _stream(stream))

    def autotune(self, stream=None) -> Tune:
        t = Tune()
        _call("shmemg_batch_autotune", self.h, _stream(stream), C.byref(t))
        return t

    def destroy(self):
        if self.h:
            _call("shmemg_batch_destroy", self.h)
            self.h = None


def batch_reduce_noalloc(descs, tile_elems=0, stream=None):
    """The batched sum reduce without any device allocation (library-held scratch)."""
    arr = (CollDesc * len(descs))(*descs)
    _call("shmemg_batch_reduce_noalloc", C.cast(arr, C.c_void_p), len(descs), tile_elems, _stream(stream))


# serving -----------------------------------------------------------------------------
class Server:
    def __init__(self, cfg: ServerCfg, stream=None):
        h = C.c_void_p(0)
        _call("shmemg_server_start", C.byref(cfg), _stream(stream), C.byref(h))
        self.h = h

    def submit(self, req: Req):
        """Returns the ticket, or None if the ring is full."""
        t = C.c_uint64(0)
        rc = lib().shmemg_server_submit(self.h, C.byref(req), C.byref(t))
        if rc == ERR_BUSY:
            return None
        if rc != SUCCESS:
            raise ShmemgError(rc, "shmemg_server_submit")
        return t.value

    def poll(self, out: np.ndarray) -> int:
        """Fills out (COMPLETION_DTYPE records) with new completions; returns how many."""
        got = C.c_int(0)
        _call("shmemg_server_poll", self.h, out.ctypes.data_as(C.c_void_p), len(out), C.byref(got))
        return got.value

    def feed(self, reqs: np.ndarray, arrival_ns: np.ndarray) -> int:
        """Submits reqs (REQ_DTYPE) at host times t0 + arrival_ns (native spin loop);
        returns t0 (CLOCK_MONOTONIC ns)."""
        reqs = np.ascontiguousarray(reqs, REQ_DTYPE)
        arr = np.ascontiguousarray(arrival_ns, np.uint64)
        t0 = C.c_uint64(0)
        _call("shmemg_server_feed", self.h, reqs.ctypes.data_as(C.c_void_p), len(reqs),
              arr.ctypes.data_as(C.c_void_p), C.byref(t0))
        return t0.value

    def stop(self):
        if self.h:
            _call("shmemg_server_stop", self.h)
            self.h = None


def device_time_ns() -> int:
    v = C.c_uint64(0)
    _call("shmemg_device_time_ns", C.byref(v))
    return v.value


def request_run(req, cfg: ServerCfg, rec_ptr: int, stream=None):
    """Plain path: one kernel for one request (REQ_DTYPE record or Req)."""
    if isinstance(req, np.ndarray):
        req = np.ascontiguousarray(req, REQ_DTYPE)
        rp = req.ctypes.data_as(C.c_void_p)
    else:
        rp = C.byref(req)
    _call("shmemg_request_run", rp, C.byref(cfg), rec_ptr, _stream(stream))


def plain_feed(reqs: np.ndarray, arrival_ns: np.ndarray, cfg: ServerCfg, recs_ptr: int, stream=None) -> int:
    """Plain path under open-loop arrivals: one kernel per request launched at its
    arrival time; completion records to recs_ptr (host-mapped). Returns t0."""
    reqs = np.ascontiguousarray(reqs, REQ_DTYPE)
    arr = np.ascontiguousarray(arrival_ns, np.uint64)
    t0 = C.c_uint64(0)
    _call("shmemg_plain_feed", reqs.ctypes.data_as(C.c_void_p), len(reqs), arr.ctypes.data_as(C.c_void_p),
          C.byref(cfg), recs_ptr, _stream(stream), C.byref(t0))
    return t0.value


def clock_offset(rounds=50):
    """(device globaltimer - host CLOCK_MONOTONIC) in ns, and its error bound."""
    off, err = C.c_int64(0), C.c_uint64(0)
    _call("shmemg_clock_offset", rounds, C.byref(off), C.byref(err))
    return off.value, err.value
