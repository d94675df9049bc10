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
