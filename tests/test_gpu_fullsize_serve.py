"""Full-size parity of the serving engine on the benchmark's workload: 512 PEs, each with
a 32 MiB page arena (16 GiB) beside its AMO table, 2^16 requests of the configuration's
mix with staged payloads -- put/get of 8 B-4 MiB, int64 AMOs on shared words, fp32 / bf16
team reductions of 64 Ki-8 Mi elements (fp32 in place; bf16 up to the largest region that
fits the arena), alltoall of 4-256 KiB per pair -- plus the largest requests of each kind
(an 8 Mi-element fp32 reduction over 64 PEs, a 64 x 256 KiB alltoall, the largest bf16
reduction, a put of half the arena), all submitted at once and served concurrently.
  * every put/get, reduction and alltoall result equals the plain launch-per-request
    path's;
  * the AMO requests' fetched values and the final words admit one serial order per word
    (the oracle's serialisation checker);
  * the largest requests and sampled ones of every non-AMO kind equal the oracle's
    result, computed on a compact heap of the request's PEs (renumbered from 0) that the
    oracle fills from the payload definition itself."""
import time

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

NPES, ARENA, NREQ = 512, 32 << 20, 1 << 16


def _drain(sg, srv, count, timeout=300.0):
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


def _largest(seed):
    """The largest staged request of each kind the arena holds."""
    n_bf = 4 * (ARENA // 28)
    while W.staged_region_bytes(16, W.FMT_BF16, n_bf, 64) > ARENA:
        n_bf -= 4
    rows = [dict(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_F32, pe=100, issuer=64, n=ARENA // 4),
            dict(kind=15, pe=300, issuer=64, n=256 << 10),
            dict(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_BF16, pe=440, issuer=64, n=n_bf),
            dict(kind=1, pe=7, issuer=500, n=ARENA // 2)]
    out = np.zeros(len(rows), W.REQ_DTYPE)
    for i, (r, kw) in enumerate(zip(out, rows)):
        r["flags"] = 1
        r["word"] = W.cb64(seed, i)
        for k, v in kw.items():
            r[k] = v
        assert W.staged_region_bytes(int(r["kind"]), int(r["fmt"]), int(r["n"]), int(r["issuer"])) <= ARENA
    return out


def _oracle_result(orc, r):
    """The oracle's result for a staged request on a compact heap of its PEs."""
    kind, pe, iss, n = int(r["kind"]), int(r["pe"]), int(r["issuer"]), int(r["n"])
    q = r.copy()
    if kind in (1, 2):
        pes = [pe] if pe == iss else [pe, iss]
        q["pe"], q["issuer"] = (0, 0) if pe == iss else (0, 1)
    else:
        pes = list(range(pe, pe + iss))
        q["pe"] = 0
    H = (W.staged_region_bytes(kind, int(r["fmt"]), n, iss) + 4095) // 4096 * 4096
    ref = orc.Heap(len(pes), H)

    def payload(seed, p, j0, count):
        return W.serve_payload_words(seed, pes[p], j0, count)
    return orc.serve_request(ref, q, 0, 1, 0, payload) & (2**64 - 1)


def test_serve_full_size(sg, orc):
    torch.cuda.set_device(0)
    lay = W.serve_layout_staged(arena_bytes=ARENA, amo_words=8192)
    heap = sg.Heap(NPES, lay.H)
    try:
        parts = heap.partitions()
        amo_init = W.cb64_torch(W.derive_seed("serve-amo"), torch.arange(NPES * lay.amo_words, device="cuda"))
        parts[:, lay.amo_offset:lay.amo_offset + 8 * lay.amo_words].view(torch.int64).copy_(
            amo_init.view(NPES, lay.amo_words))
        torch.cuda.synchronize()
        cfg = sg.ServerCfg()
        cfg.page_bytes = lay.page_bytes
        cfg.arena_offset, cfg.arena_bytes = lay.arena_offset, lay.arena_bytes
        cfg.amo_offset, cfg.amo_words = lay.amo_offset, lay.amo_words
        cfg.max_ns = 600 * 10**9
        cfg.ring_slots = 1 << 17
        big = _largest(W.derive_seed("serve-largest"))
        reqs = np.concatenate([W.gen_serve_requests(W.derive_seed("serve-reqs"), NREQ - len(big), NPES, lay,
                                                    red_hi=8 << 20, staged=True), big])
        stream = torch.cuda.Stream()
        srv = sg.Server(cfg, stream)
        srv.feed(reqs, np.zeros(NREQ, np.uint64))
        served = _drain(sg, srv, NREQ)
        srv.stop()
        assert np.all(served["status"] == 0) and np.array_equal(served["ticket"], np.arange(NREQ))
        amo_final = parts[:, lay.amo_offset:lay.amo_offset + 8 * lay.amo_words].contiguous().view(torch.int64)
        amo_final = amo_final.reshape(-1).cpu().numpy()
        amo_w0 = amo_init.cpu().numpy()
        # the plain path on the same requests (the AMO words restored first)
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
        # the largest requests and sampled ones against the oracle
        picks = list(range(NREQ - len(big), NREQ))
        for ks, k in (((1, 2), 12), ((16,), 8), ((15,), 6)):
            idx = np.nonzero(np.isin(reqs["kind"][:NREQ - len(big)], ks))[0]
            r = W.cb64_np(W.derive_seed("serve-sample"), np.arange(k, dtype=np.uint64)) % np.uint64(len(idx))
            picks += list(idx[r.astype(np.int64)])
        for i in sorted(set(int(x) for x in picks)):
            assert int(served["result"][i]) == _oracle_result(orc, reqs[i]), (i, int(reqs["kind"][i]))
    finally:
        heap.close()
