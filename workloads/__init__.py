"""Seeded synthetic inputs for the symmetric-heap workloads.

This module holds random-number generation and the *shape* of each workload (sizes,
offsets, op mixes, team layouts) and nothing of the operations' arithmetic: it never
applies a put, an atomic or a reduction.  Both the CPU oracle (``oracle/``) and the GPU
path (``paper_2607_08006_gb300``) take their inputs from here, so neither depends on the
other.

Random numbers come from the splitmix64 generator (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in two ways:

* ``SplitMix64``: a sequential stream (state += GAMMA; output = mix(state)), for the
  small, scripted workloads built in pure Python;
* ``cb64(seed, i) = mix((seed ^ i) + GAMMA)``: a counter-based draw (the first output of
  a splitmix64 stream seeded with ``seed ^ i``), vectorised over numpy or torch arrays
  for the large ones.

Zipf draws use rejection-inversion (Hoermann and Derflinger, "Rejection-inversion to
generate variates from monotone discrete distributions", 1996) in float64 on the host.
Normal draws use Box-Muller in float64 on the host (small inputs) or torch's seeded
normal generator on the device (full-size inputs, whose sampled elements are read back
as *inputs* for the oracle).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 20260701
GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


# --------------------------------------------------------------------------- splitmix64
def mix64(z: int) -> int:
    """splitmix64 output function on a Python int (64-bit wraparound)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def cb64(seed: int, i: int) -> int:
    """Counter-based draw: first splitmix64 output of the stream seeded with seed ^ i."""
    return mix64(((seed ^ i) + GAMMA) & MASK64)


def cb64_np(seed: int, idx: np.ndarray) -> np.ndarray:
    """Vectorised ``cb64`` over a numpy integer array; returns uint64."""
    with np.errstate(over="ignore"):
        z = np.array(idx, dtype=np.uint64, copy=True)   # in place from here: one temporary
        z ^= np.uint64(seed & MASK64)
        z += np.uint64(GAMMA)
        t = z >> np.uint64(30)
        z ^= t
        z *= np.uint64(_M1)
        np.right_shift(z, np.uint64(27), out=t)
        z ^= t
        z *= np.uint64(_M2)
        np.right_shift(z, np.uint64(31), out=t)
        z ^= t
        return z


def _s64(c: int) -> int:
    """A 64-bit constant as the signed int64 with the same bits."""
    c &= MASK64
    return c - (1 << 64) if c >= (1 << 63) else c


def cb64_torch(seed: int, idx):
    """``cb64`` on an int64 torch tensor (any device); the result's bits equal the
    uint64 value, stored as int64.  Logical right shifts are an arithmetic shift
    followed by a mask; multiplies wrap modulo 2^64."""
    import torch

    z = (idx.to(torch.int64) ^ _s64(seed)) + _s64(GAMMA)

    def lsr(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)

    z = (z ^ lsr(z, 30)) * _s64(_M1)
    z = (z ^ lsr(z, 27)) * _s64(_M2)
    return z ^ lsr(z, 31)


def derive_seed(tag: str, master: int = MASTER_SEED) -> int:
    """Seed of a named sub-stream: the tag's bytes folded through ``cb64``."""
    s = master & MASK64
    for b in tag.encode():
        s = cb64(s, b)
    return s


class SplitMix64:
    """Sequential splitmix64 stream with a few derived draws (pure Python)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        return mix64(self.state)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Integer in [0, n) (multiply-shift; bias < n / 2^64)."""
        return (self.next() * n) >> 64

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] inclusive."""
        return lo + self.below(hi - lo + 1)

    def log_uniform_int(self, lo: int, hi: int) -> int:
        """floor(exp(U[ln lo, ln(hi + 1)))) clamped to [lo, hi]."""
        v = int(math.floor(math.exp(math.log(lo) + self.uniform() * (math.log(hi + 1) - math.log(lo)))))
        return min(max(v, lo), hi)

    def normal(self) -> float:
        """Standard normal by Box-Muller (float64)."""
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def u01_np(bits: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from uint64 draws (top 53 bits)."""
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform_ints_np(seed: int, idx: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """int64 values in [lo, hi] from counter draws (modulo; bias < (hi-lo+1) / 2^64)."""
    span = hi - lo + 1
    return (cb64_np(seed, idx) % np.uint64(span)).astype(np.int64) + lo


def uniform_ints_torch(seed: int, idx, lo: int, hi: int):
    """Torch twin of ``uniform_ints_np``: same values, any device (int64 tensor)."""
    import torch

    z = cb64_torch(seed, idx)
    # unsigned modulo of the uint64 bit pattern: split off the top bit so the
    # dividend stays non-negative in int64 arithmetic
    span = hi - lo + 1
    hi_part = (z >> 1) & ((1 << 63) - 1)          # floor(u / 2)
    low_bit = z & 1
    r = ((hi_part % span) * 2 + low_bit) % span   # u mod span = (2*(u//2) + u%2) mod span
    return r.to(torch.int64) + lo


def normals_np(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """float64 standard normals by Box-Muller from two counter draws per value."""
    i = np.arange(offset, offset + count, dtype=np.uint64)
    u1 = 1.0 - u01_np(cb64_np(seed, 2 * i))
    u2 = u01_np(cb64_np(seed, 2 * i + 1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# --------------------------------------------------------------------------- op records
# One scripted operation = one 64-byte little-endian record.  The layout is a data
# format shared by the generator, the C ABI (shmemg_op_t) and the oracle, each of which
# declares it independently.
OP_DTYPE = np.dtype(
    [
        ("kind", "<u4"),
        ("dtype", "u1"),
        ("sub", "u1"),      # reduce op / signal op / wait comparison
        ("team", "<u2"),
        ("pe", "<i4"),      # target PE (p2p, AMO), root (broadcast)
        ("issuer", "<i4"),  # issuing PE (p2p, AMO); -1 for collectives
        ("dst", "<u8"),     # symmetric byte offset
        ("src", "<u8"),     # symmetric byte offset
        ("n", "<u8"),       # bytes (RMA, broadcast, fcollect, alltoall) or elements (reduce)
        ("operand", "<i8"),
        ("cond", "<i8"),
        ("aux", "<u8"),     # put_signal: signal word offset
    ]
)
assert OP_DTYPE.itemsize == 64

OP_PUT, OP_GET, OP_PUT_NBI, OP_GET_NBI = 1, 2, 3, 4
OP_FADD, OP_CSWAP, OP_FXOR = 5, 6, 7
OP_PUT_SIGNAL, OP_WAIT_UNTIL = 8, 9
OP_BARRIER_ALL, OP_QUIET, OP_FENCE = 10, 11, 12
OP_BCAST, OP_FCOLLECT, OP_ALLTOALL, OP_REDUCE, OP_TEAM_SYNC = 13, 14, 15, 16, 17
OP_WARP = 0x100   # flag bit of `kind`: the op is issued at warp scope (same result)
COLLECTIVE_KINDS = (OP_BARRIER_ALL, OP_BCAST, OP_FCOLLECT, OP_ALLTOALL, OP_REDUCE, OP_TEAM_SYNC)
AMO_KINDS = (OP_FADD, OP_CSWAP, OP_FXOR)

DT_INT32, DT_INT64, DT_FLOAT, DT_UINT64 = 0, 1, 2, 3
RED_SUM, RED_MAX, RED_MIN = 0, 1, 2
SIG_SET, SIG_ADD = 0, 1
CMP_EQ, CMP_NE, CMP_GT, CMP_GE, CMP_LT, CMP_LE = 0, 1, 2, 3, 4, 5
FMT_BF16, FMT_E4M3 = 0, 1


def heap_init_words(seed: int, npes: int, words_per_pe: int) -> np.ndarray:
    """Initial heap contents: word w (global index p*words_per_pe + i) = cb64(seed, w),
    returned as an int64 array of npes*words_per_pe words."""
    return cb64_np(seed, np.arange(npes * words_per_pe, dtype=np.uint64)).view(np.int64)


# --------------------------------------------------------------------------- plain script
@dataclass
class PlainScript:
    ops: np.ndarray          # OP_DTYPE records, in script order
    heap: np.ndarray         # uint8, npes * heap_bytes initial contents
    npes: int
    heap_bytes: int


class _Intervals:
    """Byte ranges touched since the last synchronising op (race-free sampling)."""

    def __init__(self):
        self.ranges = []     # (pe, lo, hi, write)
        self.amo = {}        # (pe, word offset) -> set of AMO kinds

    def clear(self):
        self.ranges.clear()
        self.amo.clear()

    def conflicts(self, pe, lo, hi, write):
        for (p, a, b, w) in self.ranges:
            if p == pe and a < hi and lo < b and (w or write):
                return True
        for (p, off) in self.amo:
            if p == pe and lo < off + 8 and off < hi:
                return True
        return False

    def add(self, pe, lo, hi, write):
        self.ranges.append((pe, lo, hi, write))

    def amo_ok(self, pe, off, kind):
        for (p, a, b, _w) in self.ranges:
            if p == pe and a < off + 8 and off < b:
                return False
        kinds = self.amo.get((pe, off))
        if kinds is None:
            return True
        # several AMOs per word per sync interval only when all are fetch_add, so that
        # the word's value at the next synchronising op does not depend on their order
        return kind == OP_FADD and kinds == {OP_FADD}

    def add_amo(self, pe, off, kind):
        self.amo.setdefault((pe, off), set()).add(kind)


def gen_plain_script(seed: int = None, npes: int = 4, heap_bytes: int = 1 << 20,
                     n_ops: int = 10000, barrier_every: int = 500, reduce_len: int = 4096,
                     bcast_bytes: int = 16384, race_free: bool = True,
                     mix=(0.30, 0.30, 0.15, 0.10, 0.075, 0.075), hot_words: int = 8) -> PlainScript:
    """The 4-PE x 1 MiB scripted stream: put/get of log-uniform 8 B-64 KiB at random
    8-byte-aligned offsets, int64 fetch_add / compare_swap on uniform targets (plus a
    small hot set for fetch_add), int64 sum reductions of ``reduce_len`` elements and
    broadcasts of ``bcast_bytes`` from a random root, with a barrier_all after every
    ``barrier_every`` ops.

    With ``race_free`` no two ops between consecutive synchronising ops (barrier or
    collective, which quiet and synchronise every PE) touch overlapping bytes with a
    write, AMO words are disjoint from every non-atomic range, and a word hit by several
    AMOs in one interval sees only fetch_add.  compare_swap's condition is the word's
    initial value with probability 1/2 (so both outcomes occur), else a random word."""
    if seed is None:
        seed = derive_seed("plain-script")
    rng = SplitMix64(seed)
    words = heap_bytes // 8
    init = heap_init_words(derive_seed("plain-heap", seed), npes, words)
    ops = []
    iv = _Intervals()
    hot = [((k * 7) % npes, ((k * 2654435761) % (words - 1)) * 8) for k in range(hot_words)]
    cum = np.cumsum(mix)

    def rec(**kw):
        r = np.zeros((), dtype=OP_DTYPE)
        r["issuer"] = -1
        for k, v in kw.items():
            r[k] = v
        return r

    def rand_range(nbytes):
        return rng.below((heap_bytes - nbytes) // 8 + 1) * 8

    for i in range(n_ops):
        u = rng.uniform()
        kind = int(np.searchsorted(cum, u, side="right"))
        kind = min(kind, len(mix) - 1)
        for _attempt in range(1000):
            if kind in (0, 1):  # put / get
                nbytes = 8 * rng.log_uniform_int(1, 8192)
                issuer = rng.below(npes)
                other = rng.below(npes)
                dst = rand_range(nbytes)
                src = rand_range(nbytes)
                if kind == 0:
                    wpe, rpe, k = other, issuer, OP_PUT
                else:
                    wpe, rpe, k = issuer, other, OP_GET
                if wpe == rpe and dst < src + nbytes and src < dst + nbytes:
                    continue
                if race_free and (iv.conflicts(wpe, dst, dst + nbytes, True)
                                  or iv.conflicts(rpe, src, src + nbytes, False)):
                    continue
                iv.add(wpe, dst, dst + nbytes, True)
                iv.add(rpe, src, src + nbytes, False)
                ops.append(rec(kind=k, pe=other, issuer=issuer, dst=dst, src=src, n=nbytes))
                break
            elif kind in (2, 3):  # fetch_add / compare_swap
                issuer = rng.below(npes)
                if kind == 2 and rng.uniform() < 0.5:
                    pe, off = hot[rng.below(len(hot))]
                else:
                    pe, off = rng.below(npes), rng.below(words) * 8
                k = OP_FADD if kind == 2 else OP_CSWAP
                if race_free and not iv.amo_ok(pe, off, k):
                    continue
                iv.add_amo(pe, off, k)
                if k == OP_FADD:
                    ops.append(rec(kind=k, dtype=DT_INT64, pe=pe, issuer=issuer, dst=off,
                                   operand=rng.randint(1, 1 << 20)))
                else:
                    if rng.uniform() < 0.5:
                        cond = int(init[pe * words + off // 8])
                    else:
                        cond = rng.next() - (1 << 63)
                    ops.append(rec(kind=k, dtype=DT_INT64, pe=pe, issuer=issuer, dst=off,
                                   operand=rng.next() - (1 << 63), cond=cond))
                break
            elif kind == 4:  # int64 sum reduce over the world team
                nb = reduce_len * 8
                src = rand_range(nb)
                dst = rand_range(nb)
                if dst < src + nb and src < dst + nb:
                    continue
                ops.append(rec(kind=OP_REDUCE, dtype=DT_INT64, sub=RED_SUM, team=0, dst=dst,
                               src=src, n=reduce_len))
                iv.clear()
                break
            else:  # broadcast over the world team from a random root
                src = rand_range(bcast_bytes)
                dst = rand_range(bcast_bytes)
                if dst < src + bcast_bytes and src < dst + bcast_bytes:
                    continue
                ops.append(rec(kind=OP_BCAST, team=0, pe=rng.below(npes), dst=dst, src=src,
                               n=bcast_bytes))
                iv.clear()
                break
        else:
            raise RuntimeError("could not place a race-free op")
        if (i + 1) % barrier_every == 0:
            ops.append(rec(kind=OP_BARRIER_ALL, team=0))
            iv.clear()
    arr = np.array(ops, dtype=OP_DTYPE) if ops else np.zeros(0, dtype=OP_DTYPE)
    return PlainScript(ops=arr, heap=init.view(np.uint8).copy(), npes=npes, heap_bytes=heap_bytes)


def sync_interval_ids(ops: np.ndarray) -> np.ndarray:
    """Index of the synchronisation interval each op belongs to (a collective or a
    barrier ends an interval and sits in an interval of its own)."""
    ids = np.zeros(len(ops), dtype=np.int64)
    cur = 0
    for i, k in enumerate(ops["kind"]):
        if k in COLLECTIVE_KINDS or k == OP_QUIET:
            cur += 1
            ids[i] = cur
            cur += 1
        else:
            ids[i] = cur
    return ids


# --------------------------------------------------------------------------- AMO stream
AMO_CODE_FADD, AMO_CODE_CSWAP, AMO_CODE_FXOR = 0, 1, 2
AMO_WORD_BITS = 27
# bijective scramble of Zipf ranks onto words (odd multiplier mod 2^27, then xor)
ZIPF_MULT = 0x5BD1E99
ZIPF_XOR = 0x2C9277B


def zipf_ranks_np(seed: int, count: int, n: int, s: float, offset: int = 0) -> np.ndarray:
    """Zipf(s) ranks in [1, n] by rejection-inversion, float64, vectorised.  Draw j of
    attempt a uses the counter (offset + j) * 64 + a, so results do not depend on
    chunking."""
    one_m_s = 1.0 - s

    def H(x):
        return np.expm1(one_m_s * np.log(x)) / one_m_s

    def Hinv(y):
        return np.exp(np.log1p(one_m_s * y) / one_m_s)

    hx1 = H(np.float64(1.5)) - 1.0
    hn = H(np.float64(n + 0.5))
    sc = 2.0 - Hinv(H(np.float64(2.5)) - 2.0 ** (-s))
    out = np.zeros(count, dtype=np.int64)
    todo = np.arange(count, dtype=np.int64)
    attempt = 0
    while todo.size:
        ctr = (todo.astype(np.uint64) + np.uint64(offset)) * np.uint64(64) + np.uint64(attempt)
        u = hn + u01_np(cb64_np(seed, ctr)) * (hx1 - hn)
        x = Hinv(u)
        k = np.clip(np.floor(x + 0.5), 1, n)
        acc = (k - x <= sc) | (u >= H(k + 0.5) - np.exp(-s * np.log(k)))
        out[todo[acc]] = k[acc].astype(np.int64)
        todo = todo[~acc]
        attempt += 1
        if attempt >= 64:
            raise RuntimeError("zipf rejection did not converge")
    return out


def amo_stream_np(seed: int, count: int, nwords_log2: int = 27, dist: str = "uniform",
                  s: float = 1.1, mix=(0.5, 0.25, 0.25), offset: int = 0,
                  only: int = None) -> np.ndarray:
    """Packed AMO ops: bits 0..26 = word index, bits 27..28 = op code (0 fetch_add,
    1 compare_swap, 2 fetch_xor).  ``only`` forces a single op code."""
    i = np.arange(offset, offset + count, dtype=np.uint64)
    mask = (1 << nwords_log2) - 1
    if dist == "uniform":
        w = (cb64_np(seed, i) & np.uint64(mask)).astype(np.uint32)
    elif dist == "zipf":
        r = zipf_ranks_np(derive_seed("zipf", seed), count, 1 << nwords_log2, s, offset)
        w = ((((r - 1).astype(np.uint64) * np.uint64(ZIPF_MULT)) & np.uint64(mask))
             ^ np.uint64(ZIPF_XOR & mask)).astype(np.uint32)
    else:
        raise ValueError(dist)
    if only is not None:
        code = np.full(count, only, dtype=np.uint32)
    else:
        u = u01_np(cb64_np(derive_seed("amo-kind", seed), i))
        code = np.where(u < mix[0], 0, np.where(u < mix[0] + mix[1], 1, 2)).astype(np.uint32)
    return w | (code << np.uint32(AMO_WORD_BITS))


# --------------------------------------------------------------------------- batched teams
@dataclass
class BatchTeams:
    start: np.ndarray   # first world rank of each team
    size: np.ndarray    # team size P_t
    n: np.ndarray       # elements per PE
    is_int: np.ndarray  # True: int64 team, else float team


def gen_batch_teams(seed: int = None, n_teams: int = 256, world: int = 128, p_lo: int = 2,
                    p_hi: int = 128, n_lo: int = 256, n_hi: int = 4 << 20,
                    int_frac: float = 0.25) -> BatchTeams:
    """Teams of contiguous ranks [start, start + P), P and n log-uniform, start uniform,
    ``int_frac`` of them int64 teams."""
    if seed is None:
        seed = derive_seed("batch-teams")
    rng = SplitMix64(seed)
    st, sz, nn, ii = [], [], [], []
    for _ in range(n_teams):
        p = rng.log_uniform_int(p_lo, min(p_hi, world))
        st.append(rng.below(world - p + 1))
        sz.append(p)
        nn.append(rng.log_uniform_int(n_lo, n_hi))
        ii.append(rng.uniform() < int_frac)
    return BatchTeams(np.array(st, np.int32), np.array(sz, np.int32), np.array(nn, np.int64),
                      np.array(ii, bool))


# --------------------------------------------------------------------------- serving
# One served request = one 64-byte record (same layout as shmemg_req_t).
REQ_DTYPE = np.dtype([("kind", "<u4"), ("dtype", "u1"), ("fmt", "u1"), ("flags", "<u2"), ("pe", "<i4"),
                      ("issuer", "<i4"), ("n", "<u8"), ("word", "<u8"), ("operand", "<i8"), ("cond", "<i8"),
                      ("src", "<u8"), ("ticket", "<u8")])
assert REQ_DTYPE.itemsize == 64
FMT_F32 = 0xFF


@dataclass
class ServeLayout:
    """Per-PE layout of a served heap: AMO table, read-only source zone, page arena."""
    H: int
    amo_offset: int
    amo_words: int
    ro_offset: int
    ro_bytes: int
    arena_offset: int
    arena_bytes: int
    page_bytes: int = 65536


def serve_layout(H: int = 32 << 20, amo_words: int = 8192) -> ServeLayout:
    amo = amo_words * 8
    half = H // 2
    return ServeLayout(H=H, amo_offset=0, amo_words=amo_words, ro_offset=amo, ro_bytes=half - amo,
                       arena_offset=half, arena_bytes=half)


def serve_layout_staged(arena_bytes: int = 32 << 20, amo_words: int = 8192) -> ServeLayout:
    """Per-PE layout for requests that stage their own payloads: the AMO table, then the
    page arena (no read-only zone)."""
    amo = amo_words * 8
    return ServeLayout(H=amo + arena_bytes, amo_offset=0, amo_words=amo_words, ro_offset=amo, ro_bytes=0,
                       arena_offset=amo, arena_bytes=arena_bytes)


def staged_region_bytes(kind: int, fmt: int, n: int, P: int) -> int:
    """Bytes of a staged request's region on each PE it touches (shmemg_req_t's staged
    payloads): the generators size requests to fit the arena with it."""
    def r16(x):
        return (x + 15) // 16 * 16
    if kind in (1, 2):
        return 2 * r16(n)
    if kind == 16:
        if fmt == FMT_BF16:
            return r16(4 * n) + r16(2 * n) + r16(4 * ((n + 127) // 128))
        return 4 * n
    if kind == 15:
        return 2 * P * n
    return 0


def serve_payload_words(seed: int, pe: int, j0: int, count: int) -> np.ndarray:
    """Words [j0, j0 + count) of PE pe's staged source part: word j holds two bfloat16
    codes b(k1) (high half) and b(k2) (low half), where k1, k2 are bytes 7 - 2q and 6 - 2q
    (q = j mod 4) of the draw cb64(seed, (pe << 40) | j // 4) -- one draw, four words --
    and b(k) = ((k & 128) << 8) | 0x3F80 | (k & 127), the bfloat16 code of
    (-1)^(k >> 7) * (1 + (k & 127) / 128)."""
    j = np.arange(j0, j0 + count, dtype=np.uint64)
    z = cb64_np(seed, (j >> np.uint64(2)) + np.uint64(pe << 40))
    sh = np.uint64(16) * (j & np.uint64(3))

    def code(k):
        k = k.astype(np.uint32)
        return ((k & np.uint32(128)) << np.uint32(8)) | np.uint32(0x3F80) | (k & np.uint32(127))
    return (code((z >> (np.uint64(56) - sh)) & np.uint64(255)) << np.uint32(16)) | \
        code((z >> (np.uint64(48) - sh)) & np.uint64(255))


def serve_source_words(seed: int, pe: int, nwords: int) -> np.ndarray:
    """Read-only source zone of one PE: binary32 words (k - 128) / 128, k = top byte of a
    counter draw -- values in [-1, 1) that are also exact in bfloat16 (low 16 bits 0)."""
    k = (cb64_np(seed, np.arange(nwords, dtype=np.uint64) + np.uint64(pe << 40)) >> np.uint64(56)).astype(np.int64)
    return ((k - 128).astype(np.float32) / np.float32(128.0))


def serve_source_words_torch(seed: int, pe: int, nwords: int, device="cuda"):
    """Torch twin of ``serve_source_words`` (same bits)."""
    import torch

    idx = torch.arange(nwords, dtype=torch.int64, device=device) + (pe << 40)
    z = cb64_torch(seed, idx)
    k = (z >> 56) & 0xFF
    return (k - 128).to(torch.float32) / 128.0


def gen_serve_requests(seed: int, count: int, npes: int, lay: ServeLayout, rma_max: int = 4 << 20,
                       red_lo: int = 1 << 16, red_hi: int = 2 << 20, a2a_lo: int = 4096, a2a_hi: int = 256 << 10,
                       p_hi: int = 64, mix=(0.60, 0.25, 0.10, 0.05), distinct_amo_words: bool = False,
                       bf16_frac: float = 0.5, staged: bool = False) -> np.ndarray:
    """Mixed served requests: put/get of 8 B..rma_max (log-uniform, multiples of 8), int64
    AMOs (fetch_add 50 %, compare_swap 25 %, fetch_xor 25 %), fp32 or bf16-payload sum
    reductions over teams of log-uniform 2..p_hi PEs with red_lo..red_hi elements, and
    alltoall of a2a_lo..a2a_hi bytes per pair (multiples of 16).
    staged=False: sources lie in the read-only zone at 16-byte aligned offsets, and
    destination footprints stay within half the arena (alltoall: P*m, reduce: 4n).
    staged=True: every non-AMO request stages its payload (flags 1, seed in `word`); its
    region must fit the arena: fp32 reductions in place (4n <= arena), bf16 ones capped at
    the largest n whose region fits, alltoall 2*P*m <= arena, put/get 2n <= arena."""
    rng = SplitMix64(seed)
    out = np.zeros(count, REQ_DTYPE)
    cum = np.cumsum(mix)
    words = npes * lay.amo_words
    amo_perm = None
    if distinct_amo_words:
        amo_perm = np.random.default_rng(seed & 0xFFFFFFFF).permutation(words)
    amo_i = 0
    ro_lo, ro_hi = lay.ro_offset, lay.ro_offset + lay.ro_bytes

    def src_off(nbytes):
        span = (ro_hi - ro_lo - nbytes) // 16
        return ro_lo + 16 * rng.below(max(span, 1))

    A = lay.arena_bytes

    def stage(r):
        r["flags"] = 1
        r["word"] = rng.next()

    for i in range(count):
        u = rng.uniform()
        r = out[i]
        if u < cum[0]:
            n = 8 * rng.log_uniform_int(1, rma_max // 8)
            r["kind"] = 1 if rng.below(2) == 0 else 2
            r["pe"], r["issuer"] = rng.below(npes), rng.below(npes)
            if staged:
                r["n"] = min(n, 8 * (A // 2 // 8))
                stage(r)
                continue
            r["n"] = n
            r["src"] = src_off(n)
        elif u < cum[1]:
            v = rng.uniform()
            r["kind"] = 5 if v < 0.5 else (6 if v < 0.75 else 7)
            r["dtype"] = DT_INT64
            if amo_perm is not None:
                r["word"] = int(amo_perm[amo_i % words])
                amo_i += 1
            else:
                r["word"] = rng.below(words)
            r["operand"] = rng.next() - (1 << 63) if r["kind"] != 5 else rng.randint(1, 1 << 20)
            r["cond"] = rng.next() - (1 << 63)
        elif u < cum[2]:
            P = rng.log_uniform_int(2, min(p_hi, npes))
            n = 4 * (rng.log_uniform_int(red_lo, red_hi) // 4)
            if not staged:
                n = min(n, (lay.arena_bytes // 2) // 4)
            bf = rng.uniform() < bf16_frac
            r["kind"] = 16
            r["dtype"] = DT_FLOAT
            r["fmt"] = FMT_BF16 if bf else FMT_F32
            r["pe"], r["issuer"] = rng.below(npes - P + 1), P
            if staged:
                n = min(n, 4 * (A // 16))
                while staged_region_bytes(16, int(r["fmt"]), n, P) > A:
                    n -= 4 * max(1, (staged_region_bytes(16, int(r["fmt"]), n, P) - A) // 28)
                r["n"] = n
                stage(r)
                continue
            r["n"] = n
            r["src"] = src_off(n * (2 if bf else 4))
            if bf:
                r["cond"] = src_off(4 * ((n + 127) // 128))
        else:
            P = rng.log_uniform_int(2, min(p_hi, npes))
            m = 16 * (rng.log_uniform_int(a2a_lo, a2a_hi) // 16)
            m = min(m, 16 * ((lay.arena_bytes // 2) // P // 16))
            r["kind"] = 15
            r["pe"], r["issuer"] = rng.below(npes - P + 1), P
            r["n"] = m
            if staged:
                stage(r)
                continue
            r["src"] = src_off(m * P)
    return out


def poisson_arrivals_ns(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Cumulative Poisson arrival times (ns) at the given rate."""
    u = 1.0 - u01_np(cb64_np(seed, np.arange(count, dtype=np.uint64)))
    gaps = -np.log(u) / rate_per_s * 1e9
    return np.cumsum(gaps).astype(np.uint64)


# --------------------------------------------------------------------------- sweep points
KiB, MiB = 1 << 10, 1 << 20
SWEEP_ELEMS = [1 << 10, 1 << 12, 1 << 14, 1 << 16, 1 << 18, 1 << 20, 1 << 22, 1 << 24]
SWEEP_A2A_BYTES = [4 * KiB, 16 * KiB, 64 * KiB, 256 * KiB, 1 * MiB]
SWEEP_BCAST_BYTES = [1 * KiB << (2 * i) for i in range(10)]
SWEEP_PUT_BYTES = [8 << (2 * i) for i in range(13)] + [256 * MiB]
