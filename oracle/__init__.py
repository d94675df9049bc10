"""CPU oracle for the symmetric-heap operations (ctypes wrapper over ``oracle.c``).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import this package.  It never imports the GPU package and
the GPU package never imports it; both take their inputs from ``workloads``.

The heap is a numpy uint8 array of npes * H bytes; PE p's partition is bytes
[p*H, (p+1)*H).  Each function applies one operation by its definition (see the C
source for the reading of the paper each follows).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P, I, U64, I64 = C.c_void_p, C.c_int, C.c_uint64, C.c_int64
            sig = {
                "or_copy": (I, [P, I, U64, I, U64, I, U64, U64]),
                "or_amo64": (I, [P, I, U64, I, I, U64, I64, I64, P]),
                "or_amo32": (I, [P, I, U64, I, I, U64, C.c_int32, C.c_int32, P]),
                "or_put_signal": (I, [P, I, U64, I, U64, I, U64, U64, U64, I, U64]),
                "or_signal_test": (I, [P, I, U64, I, U64, I, U64]),
                "or_broadcast": (I, [P, I, U64, I, I, I, U64, U64, U64, I]),
                "or_fcollect": (I, [P, I, U64, I, I, I, U64, U64, U64]),
                "or_alltoall": (I, [P, I, U64, I, I, I, U64, U64, U64]),
                "or_tree_sum_f32": (C.c_float, [P, I]),
                "or_reduce": (I, [P, I, U64, I, I, I, U64, U64, U64, I, I]),
                "or_reduce_f32_ref64": (I, [P, I, U64, I, I, I, U64, U64, P, P]),
                "or_bf16_decode": (C.c_float, [C.c_uint16]),
                "or_bf16_encode": (C.c_uint16, [C.c_float]),
                "or_e4m3_decode": (C.c_double, [C.c_uint8]),
                "or_e4m3_encode": (C.c_uint8, [C.c_float]),
                "or_quantize": (I, [P, U64, I, P, P]),
                "or_neumaier_f32": (C.c_float, [P, I]),
                "or_qsum_reduce": (I, [P, I, U64, I, I, I, U64, U64, U64, I, U64]),
                "or_qsum_ref64": (I, [P, I, U64, I, I, I, U64, U64, I, U64, P, P]),
                "or_run_script": (I, [P, I, U64, P, I64, P, I, P, P]),
                "or_cb64": (U64, [U64, U64]),
                "or_amo_stream": (I, [P, U64, P, U64, U64, U64, U64, P]),
                "or_check_serialisation": (I64, [I64, P, P, P, P, P, P, P, I, I64, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _chk(rc, what):
    if rc != 0:
        raise OracleError(f"{what}: oracle error {rc}")


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


class Heap:
    """npes partitions of H bytes, initialised from ``init`` (bytes) or zero."""

    def __init__(self, npes: int, H: int, init: np.ndarray = None):
        self.npes, self.H = npes, H
        if init is None:
            self.mem = np.zeros(npes * H, dtype=np.uint8)
        else:
            assert init.nbytes == npes * H
            self.mem = np.ascontiguousarray(init.view(np.uint8)).copy()

    def pe(self, p: int) -> np.ndarray:
        return self.mem[p * self.H:(p + 1) * self.H]

    def view(self, p: int, off: int, count: int, dtype) -> np.ndarray:
        dt = np.dtype(dtype)
        return self.pe(p)[off:off + count * dt.itemsize].view(dt)

    def _a(self):
        return (_p(self.mem), self.npes, self.H)

    # RMA (paper Sec. 2.1; blocking and _nbi forms share the final state)
    def put(self, dst, src, nbytes, pe, issuer):
        _chk(lib().or_copy(*self._a(), pe, dst, issuer, src, nbytes), "put")

    def get(self, dst, src, nbytes, pe, issuer):
        _chk(lib().or_copy(*self._a(), issuer, dst, pe, src, nbytes), "get")

    def amo64(self, kind, pe, off, v, cond=0):
        f = C.c_int64(0)
        _chk(lib().or_amo64(*self._a(), kind, pe, off, v, cond, C.byref(f)), "amo64")
        return f.value

    def amo32(self, kind, pe, off, v, cond=0):
        f = C.c_int32(0)
        _chk(lib().or_amo32(*self._a(), kind, pe, off, v, cond, C.byref(f)), "amo32")
        return f.value

    def put_signal(self, dst, src, nbytes, sig, sig_op, v, pe, issuer):
        _chk(lib().or_put_signal(*self._a(), pe, dst, issuer, src, nbytes, sig, sig_op, v),
             "put_signal")

    def signal_test(self, pe, off, cmp, v) -> bool:
        r = lib().or_signal_test(*self._a(), pe, off, cmp, v)
        if r < 0:
            raise OracleError(f"signal_test: {r}")
        return bool(r)

    # collectives over a strided team (start, stride, size)
    def broadcast(self, team, dst, src, nbytes, root):
        _chk(lib().or_broadcast(*self._a(), *team, dst, src, nbytes, root), "broadcast")

    def fcollect(self, team, dst, src, nbytes):
        _chk(lib().or_fcollect(*self._a(), *team, dst, src, nbytes), "fcollect")

    def alltoall(self, team, dst, src, m):
        _chk(lib().or_alltoall(*self._a(), *team, dst, src, m), "alltoall")

    def reduce(self, team, dst, src, nelems, dtype, op):
        _chk(lib().or_reduce(*self._a(), *team, dst, src, nelems, dtype, op), "reduce")

    def reduce_f32_ref64(self, team, src, nelems):
        y = np.zeros(nelems, np.float64)
        a = np.zeros(nelems, np.float64)
        _chk(lib().or_reduce_f32_ref64(*self._a(), *team, src, nelems, _p(y), _p(a)), "ref64")
        return y, a

    def qsum_reduce(self, team, dst, q_off, s_off, fmt, n):
        _chk(lib().or_qsum_reduce(*self._a(), *team, dst, q_off, s_off, fmt, n), "qsum_reduce")

    def qsum_ref64(self, team, q_off, s_off, fmt, n):
        y = np.zeros(n, np.float64)
        a = np.zeros(n, np.float64)
        _chk(lib().or_qsum_ref64(*self._a(), *team, q_off, s_off, fmt, n, _p(y), _p(a)), "qref64")
        return y, a

    def run_script(self, ops: np.ndarray, teams=None) -> np.ndarray:
        """Apply a scripted op list in script order; returns fetched values (AMO ops)."""
        ops = np.ascontiguousarray(ops)
        assert ops.dtype.itemsize == 64
        if teams is None:
            teams = [(0, 1, self.npes)]
        t = np.ascontiguousarray(np.array(teams, dtype=np.int32).reshape(-1))
        fetched = np.zeros(len(ops), np.int64)
        bad = C.c_int64(-1)
        rc = lib().or_run_script(*self._a(), _p(ops), len(ops), _p(t), len(t) // 3, _p(fetched),
                                 C.byref(bad))
        if rc != 0:
            raise OracleError(f"run_script: error {rc} at op {bad.value}")
        return fetched


def tree_sum_f32(values) -> np.float32:
    v = np.ascontiguousarray(np.array(values, dtype=np.float32))
    return np.float32(lib().or_tree_sum_f32(_p(v), len(v)))


def neumaier_f32(values) -> np.float32:
    v = np.ascontiguousarray(np.array(values, dtype=np.float32))
    return np.float32(lib().or_neumaier_f32(_p(v), len(v)))


def bf16_encode(x: float) -> int:
    return int(lib().or_bf16_encode(float(np.float32(x))))


def bf16_decode(q: int) -> float:
    return float(lib().or_bf16_decode(q))


def e4m3_encode(x: float) -> int:
    return int(lib().or_e4m3_encode(float(np.float32(x))))


def e4m3_decode(q: int) -> float:
    return float(lib().or_e4m3_decode(q))


def quantize(x: np.ndarray, fmt: int):
    """Per-128-element block quantisation of one PE's floats -> (codes, scales)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n = len(x)
    q = np.zeros(n, np.uint8 if fmt == 1 else np.uint16)
    s = np.zeros((n + 127) // 128, np.float32)
    _chk(lib().or_quantize(_p(x), n, fmt, _p(q), _p(s)), "quantize")
    return q, s


def checksum32(buf: np.ndarray) -> int:
    """Result encoding of a served request's output: sum over its little-endian 32-bit
    words w_i of w_i * (2i + 1), modulo 2^64."""
    w = np.frombuffer(np.ascontiguousarray(buf).tobytes(), dtype="<u4").astype(np.uint64)
    i = np.arange(len(w), dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(w * (np.uint64(2) * i + np.uint64(1)), dtype=np.uint64))


def serve_request(heap: "Heap", r, amo_offset: int, amo_words: int, scratch_off: int, payload=None):
    """Expected result of one served request applied alone to `heap` (its output is built
    at scratch_off): the fetched value for an AMO, else the output's checksum32.  A request
    that stages its payload (flags bit 0) builds its whole region at scratch_off; the
    caller's payload(seed, pe, j0, count) gives words [j0, j0 + count) of heap PE pe's
    source part."""
    kind = int(r["kind"])
    if int(r["flags"]) & 1:
        return _serve_staged(heap, r, scratch_off, payload)
    if kind in (5, 6, 7):
        w = int(r["word"])
        return heap.amo64(kind, w // amo_words, amo_offset + 8 * (w % amo_words), int(r["operand"]), int(r["cond"]))
    pe, iss, n, src = int(r["pe"]), int(r["issuer"]), int(r["n"]), int(r["src"])
    if kind in (1, 2):
        sp, dp = (iss, pe) if kind == 1 else (pe, iss)
        heap.put(scratch_off, src, n, dp, sp)
        return checksum32(heap.pe(dp)[scratch_off:scratch_off + n])
    team = (pe, 1, iss)
    if kind == 16:
        if int(r["dtype"]) == 1:
            heap.reduce(team, scratch_off, src, n, 1, 0)
            nb = 8 * n
        elif int(r["fmt"]) == 0:
            heap.qsum_reduce(team, scratch_off, src, int(r["cond"]), 0, n)
            nb = 4 * n
        else:
            heap.reduce(team, scratch_off, src, n, 2, 0)
            nb = 4 * n
        return checksum32(heap.pe(pe)[scratch_off:scratch_off + nb])
    if kind == 15:
        heap.alltoall(team, scratch_off, src, n)
        return checksum32(np.concatenate([heap.pe(pe + j)[scratch_off:scratch_off + iss * n] for j in range(iss)]))
    raise ValueError(kind)


def _serve_staged(heap: "Heap", r, R: int, payload):
    """A request with a staged payload, region at offset R of every PE it touches (the
    request record's layout): the source part is written word by word from the payload
    function, then the operation runs on it by its definition."""
    kind, pe, iss, n, seed = int(r["kind"]), int(r["pe"]), int(r["issuer"]), int(r["n"]), int(r["word"])

    def r16(x):
        return (x + 15) // 16 * 16

    def write(p, part, j0, count):
        heap.pe(p)[part + 4 * j0:part + 4 * (j0 + count)] = np.asarray(payload(seed, p, j0, count), np.uint32).view(np.uint8)

    if kind in (1, 2):
        a = r16(n)
        sp, dp = (iss, pe) if kind == 1 else (pe, iss)
        write(sp, R + a, 0, n // 4)
        heap.put(R, R + a, n, dp, sp)                 # destination part on dp <- source part on sp
        return checksum32(heap.pe(dp)[R:R + n])
    team = (pe, 1, iss)
    if kind == 16:
        dt, fmt = int(r["dtype"]), int(r["fmt"])
        if dt == 1:                                   # int64, in place
            for p in range(pe, pe + iss):
                write(p, R, 0, 2 * n)
            heap.reduce(team, R, R, n, 1, 0)
            return checksum32(heap.pe(pe)[R:R + 8 * n])
        if fmt == 0:                                  # bf16 codes and per-128 scales after the fp32 output
            c4, c2 = r16(4 * n), r16(2 * n)
            for p in range(pe, pe + iss):
                write(p, R + c4, 0, n // 2)
                write(p, R + c4, c2 // 4, (n + 127) // 128)
            heap.qsum_reduce(team, R, R + c4, R + c4 + c2, 0, n)
        else:                                         # fp32, in place
            for p in range(pe, pe + iss):
                write(p, R, 0, n)
            heap.reduce(team, R, R, n, 2, 0)
        return checksum32(heap.pe(pe)[R:R + 4 * n])
    if kind == 15:
        for p in range(pe, pe + iss):
            write(p, R + iss * n, 0, iss * n // 4)
        heap.alltoall(team, R, R + iss * n, n)
        return checksum32(np.concatenate([heap.pe(pe + j)[R:R + iss * n] for j in range(iss)]))
    raise ValueError(kind)


def cb64(seed: int, i: int) -> int:
    return int(lib().or_cb64(seed, i))


def amo_stream(table: np.ndarray, ops: np.ndarray, op_seed: int, table_seed: int,
               first_op: int = 0, want_fetched: bool = True):
    """Apply a packed AMO stream sequentially to ``table`` (int64, modified in place)."""
    assert table.dtype == np.int64 and ops.dtype == np.uint32
    fetched = np.zeros(len(ops), np.int64) if want_fetched else None
    _chk(lib().or_amo_stream(_p(table), len(table), _p(ops), len(ops), first_op, op_seed,
                             table_seed, _p(fetched) if want_fetched else None), "amo_stream")
    return fetched


def _splitmix64_np(seed: int, i: np.ndarray) -> np.ndarray:
    """splitmix64 (Steele, Lea, Flood, OOPSLA 2014): first output of the stream seeded
    with seed ^ i, vectorised (uint64 arithmetic wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) ^ i.astype(np.uint64)) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def amo_add_word_sums(ops: np.ndarray, first_op: int, op_seed: int, words: np.ndarray) -> np.ndarray:
    """For each word of the sorted array ``words``: the sum of the fetch_add operands
    ((r mod 2^20) + 1, r = splitmix64(op_seed ^ i)) of the ops among ``ops`` (packed, op i
    = first_op + position) that target it.  Fetch_adds commute (Sec. 2.1 atomics), so a
    word that only fetch_adds touch ends at its initial value plus this sum in any
    serial order.  Sums of up to 2^32 operands stay below 2^53, exact in binary64."""
    if len(words) == 0:
        return np.zeros(0, np.int64)
    w = (ops & np.uint32((1 << 27) - 1)).astype(np.int64)
    code = ops >> np.uint32(27)
    pos = np.searchsorted(words, w)
    pos[pos == len(words)] = 0
    hit = (words[pos] == w) & (code == 0)
    i = np.nonzero(hit)[0]
    r = _splitmix64_np(op_seed, i.astype(np.uint64) + np.uint64(first_op))
    v = (r & np.uint64((1 << 20) - 1)) + np.uint64(1)
    return np.bincount(pos[i], weights=v.astype(np.float64), minlength=len(words)).astype(np.int64)


def check_serialisation(group, kind, operand, cond, fetched, w0, final=None,
                        budget_per_group: int = 1 << 26):
    """Number of word groups whose fetched values admit no valid serial order (0 = all
    valid); -1 if the search was inconclusive.  Arrays are per op."""
    n = len(kind)
    group = np.ascontiguousarray(group, np.int64)
    kind = np.ascontiguousarray(kind, np.int32)
    operand = np.ascontiguousarray(operand, np.int64)
    cond = np.ascontiguousarray(cond, np.int64)
    fetched = np.ascontiguousarray(fetched, np.int64)
    w0 = np.ascontiguousarray(w0, np.int64)
    has_final = final is not None
    fin = np.ascontiguousarray(final if has_final else np.zeros(n), np.int64)
    bad = C.c_int64(-1)
    r = lib().or_check_serialisation(n, _p(group), _p(kind), _p(operand), _p(cond), _p(fetched),
                                     _p(w0), _p(fin), int(has_final), budget_per_group, C.byref(bad))
    return int(r)


def halo_jacobi(grid, iters: int) -> np.ndarray:
    """Jacobi sweeps on a periodic 2-D binary32 grid: every point becomes
    0.25 * ((up + down) + (left + right)), each operation rounded to binary32 -- the
    stencil of the halo-exchange workload (paper Sec. 4.4, case study 1), written on the
    whole grid, with no decomposition into tiles and no halos."""
    g = np.ascontiguousarray(grid, dtype=np.float32)
    q = np.float32(0.25)
    for _ in range(iters):
        up, dn = np.roll(g, 1, axis=0), np.roll(g, -1, axis=0)
        lf, rt = np.roll(g, 1, axis=1), np.roll(g, -1, axis=1)
        g = q * ((up + dn) + (lf + rt))
    return g

