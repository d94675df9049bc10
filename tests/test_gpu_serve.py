"""Serving engine: results of mixed, concurrently served requests equal their results
alone, the plain launch-per-request path's results, and the oracle's; admission errors
and bounded exit."""
import time

import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import upload

pytestmark = pytest.mark.gpu

NPES, H = 32, 8 << 20


def _layout():
    return W.serve_layout(H=H, amo_words=4096)


def _init(lay, seed=11):
    init = np.zeros((NPES, H), np.uint8)
    init[:, :lay.amo_words * 8] = W.cb64_np(seed, np.arange(NPES * lay.amo_words, dtype=np.uint64)).view(
        np.uint8).reshape(NPES, -1)
    for p in range(NPES):
        init[p, lay.ro_offset:lay.ro_offset + lay.ro_bytes] = W.serve_source_words(seed, p, lay.ro_bytes // 4).view(np.uint8)
    return init.reshape(-1)


def _cfg(sg, lay, **kw):
    c = sg.ServerCfg()
    c.page_bytes = lay.page_bytes
    c.arena_offset, c.arena_bytes = lay.arena_offset, lay.arena_bytes
    c.amo_offset, c.amo_words = lay.amo_offset, lay.amo_words
    c.max_ns = 120 * 10**9
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _requests(lay, count=1200, seed=3):
    return W.gen_serve_requests(seed, count, NPES, lay, rma_max=256 << 10, red_lo=1024, red_hi=1 << 16,
                                a2a_lo=16, a2a_hi=16 << 10, p_hi=16, distinct_amo_words=True)


def _drain(sg, srv, count, timeout=60.0):
    out = np.zeros(count, sg.COMPLETION_DTYPE)
    buf = np.zeros(4096, sg.COMPLETION_DTYPE)
    got, t0 = 0, time.time()
    while got < count:
        k = srv.poll(buf)
        out[got:got + k] = buf[:k]
        got += k
        if k == 0:
            assert time.time() - t0 < timeout, f"only {got}/{count} completions"
            time.sleep(0.0005)
    return out


def _by_ticket(recs):
    o = np.argsort(recs["ticket"])
    return recs[o]


def test_served_results_invariant_alone_mix_plain_oracle(sg, heapf, orc):
    lay = _layout()
    h = heapf(NPES, H)
    init = _init(lay)
    reqs = _requests(lay)
    cfg = _cfg(sg, lay)
    # ---- mixed: everything submitted at once, served concurrently
    upload(h, init)
    stream = torch.cuda.Stream()
    srv = sg.Server(cfg, stream)
    srv.feed(reqs, np.zeros(len(reqs), np.uint64))
    mix = _by_ticket(_drain(sg, srv, len(reqs)))
    srv.stop()
    amo_after_mix = h.partitions()[:, :lay.amo_words * 8].cpu().numpy()
    assert np.all(mix["status"] == 0), np.unique(mix["status"])
    assert np.array_equal(mix["ticket"], np.arange(len(reqs)))
    # continuous batching: requests overlapped in time on the device
    ev = sorted([(int(a), 1) for a in mix["t_admit_ns"]] + [(int(d), -1) for d in mix["t_done_ns"]])
    depth, peak = 0, 0
    for _, d in ev:
        depth += d
        peak = max(peak, depth)
    assert peak >= 2
    # ---- alone: one request at a time through the same server
    upload(h, init)
    srv = sg.Server(cfg, stream)
    alone = np.zeros(len(reqs), sg.COMPLETION_DTYPE)
    for i in range(len(reqs)):
        srv.feed(reqs[i:i + 1], np.zeros(1, np.uint64))
        alone[i] = _drain(sg, srv, 1)[0]
    srv.stop()
    assert np.all(alone["status"] == 0)
    assert np.array_equal(alone["result"], mix["result"])
    # ---- plain path: one kernel per request
    upload(h, init)
    recs = torch.zeros(len(reqs) * sg.COMPLETION_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    sg.plain_feed(reqs, np.zeros(len(reqs), np.uint64), cfg, recs.data_ptr(), stream)
    stream.synchronize()
    plain = np.frombuffer(recs.numpy().tobytes(), sg.COMPLETION_DTYPE)
    assert np.all(plain["seq"] == 1) and np.all(plain["status"] == 0)
    assert np.array_equal(plain["result"], mix["result"])
    # ---- oracle, request by request on the same initial heap
    ref = orc.Heap(NPES, H, init)
    want = np.array([orc.serve_request(ref, r, lay.amo_offset, lay.amo_words, lay.arena_offset) & (2**64 - 1)
                     for r in reqs], dtype=np.uint64)
    assert np.array_equal(mix["result"], want)
    assert np.array_equal(amo_after_mix.reshape(-1), ref.mem.reshape(NPES, H)[:, :lay.amo_words * 8].reshape(-1))


def test_server_admission_errors_and_idle_exit(sg, heapf):
    lay = _layout()
    h = heapf(NPES, H)
    upload(h, _init(lay))
    cfg = _cfg(sg, lay, idle_ns=200_000_000)
    bad = np.zeros(3, sg.REQ_DTYPE)
    bad[0] = (1, 0, 0, 0, 99, 0, 64, 0, 0, 0, lay.ro_offset, 0)                 # PE out of range
    bad[1] = (15, 0, 0, 0, 0, 32, lay.arena_bytes // 16, 0, 0, 0, lay.ro_offset, 0)  # bigger than the arena
    bad[2] = (1, 0, 0, 0, 1, 0, 64, 0, 0, 0, lay.ro_offset, 0)                  # fine
    stream = torch.cuda.Stream()
    srv = sg.Server(cfg, stream)
    srv.feed(bad, np.zeros(3, np.uint64))
    got = _by_ticket(_drain(sg, srv, 3))
    assert list(got["status"]) == [sg.ERR_INVALID_ARG, sg.ERR_INVALID_ARG, 0] or \
        list(got["status"]) == [sg.ERR_INVALID_ARG, sg.ERR_OUT_OF_HEAP, 0]
    time.sleep(0.5)                          # idle bound: the kernel leaves by itself
    assert stream.query()
    srv.stop()


def _staged_requests(lay, npes, count=600, seed=5):
    """The generator's staged mix plus the boundary cases of the staged layout: an fp32
    reduction in place over the whole arena, the largest bf16 reduction that fits, an
    alltoall whose source and destination blocks fill the arena, a self put and a put of
    half the arena, a get whose size is not a multiple of 16, an int64 reduction."""
    reqs = W.gen_serve_requests(seed, count, npes, lay, rma_max=256 << 10, red_lo=1024, red_hi=1 << 16,
                                a2a_lo=16, a2a_hi=16 << 10, p_hi=16, distinct_amo_words=True, staged=True)
    A = lay.arena_bytes
    extra = np.zeros(8, W.REQ_DTYPE)
    n_bf = 4 * (A // 28)
    while W.staged_region_bytes(16, W.FMT_BF16, n_bf, 5) > A:
        n_bf -= 4
    rows = [dict(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_F32, pe=3, issuer=8, n=A // 4),
            dict(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_BF16, pe=20, issuer=5, n=n_bf),
            dict(kind=15, pe=9, issuer=16, n=A // 32),
            dict(kind=1, pe=7, issuer=7, n=4096),
            dict(kind=1, pe=2, issuer=30, n=A // 2),
            dict(kind=2, pe=11, issuer=4, n=1000),
            dict(kind=16, dtype=W.DT_INT64, fmt=0, pe=25, issuer=3, n=5000),
            dict(kind=2, pe=31, issuer=31, n=8)]
    for r, kw in zip(extra, rows):
        r["flags"] = 1
        r["word"] = W.cb64(seed, int(kw["n"]) ^ (kw["pe"] << 32))
        for k, v in kw.items():
            r[k] = v
    for r in extra:
        assert W.staged_region_bytes(int(r["kind"]), int(r["fmt"]), int(r["n"]), int(r["issuer"])) <= A
    return np.concatenate([extra[:4], reqs, extra[4:]])


def test_staged_served_results_invariant_alone_mix_plain_oracle(sg, heapf, orc):
    """Requests that stage their own payload (fp32 reductions in place, up to whole-arena
    regions): served concurrently, one at a time, on the plain path and by the oracle,
    the results agree; the AMO table ends as the oracle's."""
    lay = W.serve_layout_staged(arena_bytes=4 << 20, amo_words=4096)
    Hs = lay.H
    h = heapf(NPES, Hs)
    init = np.zeros((NPES, Hs), np.uint8)
    init[:, :lay.amo_words * 8] = W.cb64_np(17, np.arange(NPES * lay.amo_words, dtype=np.uint64)).view(
        np.uint8).reshape(NPES, -1)
    init = init.reshape(-1)
    reqs = _staged_requests(lay, NPES)
    cfg = _cfg(sg, lay)
    stream = torch.cuda.Stream()
    upload(h, init)
    srv = sg.Server(cfg, stream)
    srv.feed(reqs, np.zeros(len(reqs), np.uint64))
    mix = _by_ticket(_drain(sg, srv, len(reqs)))
    srv.stop()
    amo_after_mix = h.partitions()[:, :lay.amo_words * 8].cpu().numpy()
    assert np.all(mix["status"] == 0), np.unique(mix["status"], return_counts=True)
    upload(h, init)
    srv = sg.Server(cfg, stream)
    alone = np.zeros(len(reqs), sg.COMPLETION_DTYPE)
    for i in range(len(reqs)):
        srv.feed(reqs[i:i + 1], np.zeros(1, np.uint64))
        alone[i] = _drain(sg, srv, 1)[0]
    srv.stop()
    assert np.all(alone["status"] == 0)
    assert np.array_equal(alone["result"], mix["result"])
    upload(h, init)
    recs = torch.zeros(len(reqs) * sg.COMPLETION_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    sg.plain_feed(reqs, np.zeros(len(reqs), np.uint64), cfg, recs.data_ptr(), stream)
    stream.synchronize()
    plain = np.frombuffer(recs.numpy().tobytes(), sg.COMPLETION_DTYPE)
    assert np.all(plain["seq"] == 1) and np.all(plain["status"] == 0)
    assert np.array_equal(plain["result"], mix["result"])
    ref = orc.Heap(NPES, Hs, init)
    want = np.array([orc.serve_request(ref, r, lay.amo_offset, lay.amo_words, lay.arena_offset, W.serve_payload_words)
                     & (2**64 - 1) for r in reqs], dtype=np.uint64)
    bad = np.nonzero(mix["result"] != want)[0]
    assert len(bad) == 0, [(int(i), int(reqs["kind"][i]), int(reqs["n"][i])) for i in bad[:10]]
    assert np.array_equal(amo_after_mix.reshape(-1), ref.mem.reshape(NPES, Hs)[:, :lay.amo_words * 8].reshape(-1))


def test_staged_admission_refuses_regions_beyond_the_arena(sg, heapf):
    lay = W.serve_layout_staged(arena_bytes=1 << 20, amo_words=1024)
    h = heapf(4, lay.H)
    cfg = _cfg(sg, lay, idle_ns=200_000_000)
    bad = np.zeros(4, sg.REQ_DTYPE)
    for r, kw in zip(bad, [dict(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_F32, pe=0, issuer=2, n=(1 << 18) + 4),  # 4n > arena
                           dict(kind=15, pe=0, issuer=4, n=(1 << 17) + 16),                                   # 2Pm > arena
                           dict(kind=5, dtype=W.DT_INT64, word=3, operand=1),                                 # AMOs never stage
                           dict(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_F32, pe=0, issuer=4, n=1 << 18)]):       # exactly fits
        r["flags"] = 1
        for k, v in kw.items():
            r[k] = v
    stream = torch.cuda.Stream()
    srv = sg.Server(cfg, stream)
    srv.feed(bad, np.zeros(len(bad), np.uint64))
    got = _by_ticket(_drain(sg, srv, len(bad)))
    srv.stop()
    assert list(got["status"]) == [sg.ERR_OUT_OF_HEAP, sg.ERR_OUT_OF_HEAP, sg.ERR_INVALID_ARG, 0]


def test_staged_ragged_and_degenerate_requests(sg, heapf, orc):
    """Staged requests at ragged and degenerate sizes: reductions of 4..8188 elements (a
    ragged last tile, a ragged last 128-element block for bf16 scales, one-member teams),
    puts and gets of 8 B and of one RMA tile plus 8 B, self puts, alltoalls of 16 B and of
    one chunk plus 16 B per pair with teams of 1-3; each result alone = plain = oracle."""
    npes = 8
    lay = W.serve_layout_staged(arena_bytes=2 << 20, amo_words=256)
    h = heapf(npes, lay.H)
    init = np.zeros(npes * lay.H, np.uint8)
    rows = []
    for n in (4, 12, 20, 124, 132, 8188, 8196):
        for fmt, dt in ((W.FMT_F32, W.DT_FLOAT), (W.FMT_BF16, W.DT_FLOAT), (0, W.DT_INT64)):
            for P in (1, 3):
                rows.append(dict(kind=16, dtype=dt, fmt=fmt, pe=npes - P, issuer=P, n=n))
    for n in (8, 24, (64 << 10) + 8):
        rows += [dict(kind=1, pe=2, issuer=5, n=n), dict(kind=2, pe=6, issuer=1, n=n), dict(kind=1, pe=3, issuer=3, n=n)]
    for m in (16, 48, (32 << 10) + 16):
        for P in (1, 2, 3):
            rows.append(dict(kind=15, pe=1, issuer=P, n=m))
    reqs = np.zeros(len(rows), W.REQ_DTYPE)
    for i, (r, kw) in enumerate(zip(reqs, rows)):
        r["flags"] = 1
        r["word"] = W.cb64(77, i)
        for k, v in kw.items():
            r[k] = v
    cfg = _cfg(sg, lay)
    stream = torch.cuda.Stream()
    upload(h, init)
    srv = sg.Server(cfg, stream)
    alone = np.zeros(len(reqs), sg.COMPLETION_DTYPE)
    for i in range(len(reqs)):
        srv.feed(reqs[i:i + 1], np.zeros(1, np.uint64))
        alone[i] = _drain(sg, srv, 1)[0]
    srv.stop()
    assert np.all(alone["status"] == 0), [(rows[i], int(alone["status"][i])) for i in np.nonzero(alone["status"])[0][:5]]
    recs = torch.zeros(len(reqs) * sg.COMPLETION_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    sg.plain_feed(reqs, np.zeros(len(reqs), np.uint64), cfg, recs.data_ptr(), stream)
    stream.synchronize()
    plain = np.frombuffer(recs.numpy().tobytes(), sg.COMPLETION_DTYPE)
    assert np.all(plain["status"] == 0)
    assert np.array_equal(plain["result"], alone["result"])
    ref = orc.Heap(npes, lay.H, init)
    want = np.array([orc.serve_request(ref, r, lay.amo_offset, lay.amo_words, lay.arena_offset, W.serve_payload_words)
                     & (2**64 - 1) for r in reqs], dtype=np.uint64)
    bad = np.nonzero(alone["result"] != want)[0]
    assert len(bad) == 0, [rows[i] for i in bad[:8]]
