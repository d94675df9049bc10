"""Full-size parity of the serving engine on the benchmark's workload: 512 PEs x 32 MiB,
2^16 requests of the configuration's mix (put/get of 8 B-4 MiB, int64 AMOs on shared
words, fp32 / bf16 team reductions of up to 2 Mi elements, alltoall of up to 256 KiB per
pair), all submitted at once and served concurrently.
  * every put/get, reduction and alltoall result equals the plain launch-per-request
    path's;
  * the AMO requests' fetched values and the final words admit one serial order per word
    (the oracle's serialisation checker);
  * sampled requests of every non-AMO kind equal the oracle's result, computed on a
    compact heap that holds only the bytes the request reads (its PEs renumbered from 0,
    its sources moved to offset 0)."""
import time

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

NPES, HS, NREQ = 512, 32 << 20, 1 << 16


def _drain(sg, srv, count, timeout=120.0):
    out = np.zeros(count, sg.COMPLETION_DTYPE)
    buf = np.zeros(16384, sg.COMPLETION_DTYPE)
    got, t0 = 0, time.time()
    while got < count:
        k = srv.poll(buf)
        out[got:got + k] = buf[:k]
        got += k
        if k == 0:
            assert time.time() - t0 < timeout, f"only {got}/{count} completions"
            time.sleep(0.0002)
    return out[np.argsort(out["ticket"])]


def _compact(parts, r):
    """(oracle heap inputs, rewritten request, scratch offset): the request's PEs as 0..k-1,
    its source bytes at offset 0 of each, the output built above them."""
    kind, pe, iss, n, src = int(r["kind"]), int(r["pe"]), int(r["issuer"]), int(r["n"]), int(r["src"])
    q = r.copy()
    if kind in (1, 2):
        sp = iss if kind == 1 else pe
        pes = [sp] if pe == iss else ([iss, pe])
        spans = [(src, n)]
        q["issuer"], q["pe"] = (0, 0) if pe == iss else (0, 1)
    else:
        pes = list(range(pe, pe + iss))
        q["pe"] = 0
        if kind == 16 and int(r["fmt"]) == 0:
            spans = [(src, 2 * n), (int(r["cond"]), 4 * ((n + 127) // 128))]
        elif kind == 16:
            spans = [(src, 4 * n)]
        else:
            spans = [(src, iss * n)]
    offs, o = [], 0
    for _, ln in spans:
        offs.append(o)
        o = (o + ln + 255) // 256 * 256
    q["src"] = offs[0]
    if len(spans) > 1:
        q["cond"] = offs[1]
    out_bytes = {1: n, 2: n, 15: iss * n, 16: 4 * n}[kind]
    scratch = o
    H = (scratch + out_bytes + 4095) // 4096 * 4096
    mem = np.zeros((len(pes), H), np.uint8)
    for i, p in enumerate(pes):
        for (s0, ln), d0 in zip(spans, offs):
            mem[i, d0:d0 + ln] = parts[p, s0:s0 + ln].cpu().numpy()
    return len(pes), H, mem.reshape(-1), q, scratch


def test_serve_full_size(sg, orc):
    torch.cuda.set_device(0)
    lay = W.serve_layout(H=HS, amo_words=8192)
    heap = sg.Heap(NPES, HS)
    try:
        parts = heap.partitions()
        seed = W.derive_seed("serve-inputs")
        for p in range(NPES):
            parts[p, lay.ro_offset:lay.ro_offset + lay.ro_bytes].view(torch.float32).copy_(
                W.serve_source_words_torch(seed, p, lay.ro_bytes // 4))
        amo_init = W.cb64_torch(W.derive_seed("serve-amo"), torch.arange(NPES * lay.amo_words, device="cuda"))
        parts[:, lay.amo_offset:lay.amo_offset + 8 * lay.amo_words].view(torch.int64).copy_(
            amo_init.view(NPES, lay.amo_words))
        torch.cuda.synchronize()
        cfg = sg.ServerCfg()
        cfg.page_bytes = lay.page_bytes
        cfg.arena_offset, cfg.arena_bytes = lay.arena_offset, lay.arena_bytes
        cfg.amo_offset, cfg.amo_words = lay.amo_offset, lay.amo_words
        cfg.max_ns = 300 * 10**9
        cfg.ring_slots = 1 << 17
        reqs = W.gen_serve_requests(W.derive_seed("serve-reqs"), NREQ, NPES, lay)
        stream = torch.cuda.Stream()
        srv = sg.Server(cfg, stream)
        srv.feed(reqs, np.zeros(NREQ, np.uint64))
        served = _drain(sg, srv, NREQ)
        srv.stop()
        assert np.all(served["status"] == 0) and np.array_equal(served["ticket"], np.arange(NREQ))
        amo_final = parts[:, lay.amo_offset:lay.amo_offset + 8 * lay.amo_words].contiguous().view(torch.int64)
        amo_final = amo_final.reshape(-1).cpu().numpy()
        amo_w0 = amo_init.cpu().numpy()
        # the plain path on the same inputs (the AMO words restored first)
        parts[:, lay.amo_offset:lay.amo_offset + 8 * lay.amo_words].view(torch.int64).copy_(
            amo_init.view(NPES, lay.amo_words))
        recs = torch.zeros(NREQ * sg.COMPLETION_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        sg.plain_feed(reqs, np.zeros(NREQ, np.uint64), cfg, recs.data_ptr(), stream)
        stream.synchronize()
        plain = np.frombuffer(recs.numpy().tobytes(), sg.COMPLETION_DTYPE)
        assert np.all(plain["status"] == 0)
        is_amo = np.isin(reqs["kind"], (5, 6, 7))
        assert np.array_equal(served["result"][~is_amo], plain["result"][~is_amo])
        # AMOs: one serial order per word
        a = np.nonzero(is_amo)[0]
        w = reqs["word"][a].astype(np.int64)
        got = orc.check_serialisation(w, reqs["kind"][a].astype(np.int32), reqs["operand"][a], reqs["cond"][a],
                                      served["result"][a].view(np.int64), amo_w0[w], amo_final[w])
        assert got == 0 and len(a) > 10000
        # sampled requests against the oracle
        picks = []
        for ks, k in (((1, 2), 20), ((16,), 20), ((15,), 8)):
            idx = np.nonzero(np.isin(reqs["kind"], ks))[0]
            order = np.argsort(-reqs["n"][idx].astype(np.int64) * np.maximum(reqs["issuer"][idx], 1))
            picks += list(idx[order[:2]])   # the largest of the kind
            r = W.cb64_np(W.derive_seed("serve-sample"), np.arange(k, dtype=np.uint64)) % np.uint64(len(idx))
            picks += list(idx[r.astype(np.int64)])
        for i in sorted(set(int(x) for x in picks)):
            npe, H, mem, q, scratch = _compact(parts, reqs[i])
            ref = orc.Heap(npe, H, mem)
            want = orc.serve_request(ref, q, 0, 1, scratch) & (2**64 - 1)
            assert int(served["result"][i]) == want, (i, int(reqs["kind"][i]))
    finally:
        heap.close()
