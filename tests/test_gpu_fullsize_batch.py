"""Full-size parity of the batched engine on the benchmark's own workload (256 teams of
2-128 PEs over a 128-PE heap, n up to 4 Mi, 25 % int64 teams), fp32 and bf16 / E4M3
payloads, graph-captured and autotuned as the benchmark times it.  Sampled 128-element
blocks of sampled teams are compared bitwise with the oracle run on a small heap that
holds only those blocks (every member's inputs, with the blocks' scales)."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

BLOCKS = 3   # sampled 128-element blocks per team


@pytest.fixture(scope="module")
def wl(sg):
    import bench

    torch.cuda.set_device(0)
    w = bench.BatchWorkload(torch, sg)
    yield w
    w.close()


def _blocks(t, n):
    nb = (n + 127) // 128
    r = W.cb64_np(W.derive_seed("batch-sample") ^ t, np.arange(BLOCKS, dtype=np.uint64))
    b = np.unique((r % np.uint64(nb)).astype(np.int64))
    return b   # ascending: a partial last block of the team comes last


def _elems(blocks, n):
    return np.concatenate([np.arange(128 * b, min(128 * b + 128, n)) for b in blocks])


@pytest.mark.parametrize("fmt", [-1, 0, 1])
def test_batch_full_size_sampled_blocks(sg, orc, wl, fmt):
    if fmt >= 0:
        wl.quantize(fmt)
    b = sg.Batch(wl.descs(fmt), sg.Tune(16384, 0, 0, 0))
    try:
        b.autotune()
        b.launch()
        torch.cuda.synchronize()
        assert sg.get_status()[0] == 0
        teams = list(range(0, len(wl.P), 7)) + [int(np.argmax(wl.P * wl.n))]
        for t in teams:
            k, src, dst, codes, sc = wl.lay[t]
            P, n, st0 = int(wl.P[t]), int(wl.n[t]), int(wl.bt.start[t])
            blocks = _blocks(t, n)
            el = _elems(blocks, n)
            m = len(el)
            ix = torch.from_numpy(el).cuda()
            members = range(st0, st0 + P)
            if k == "i64":
                x = np.stack([wl.heap.view(src, p, torch.int64, n)[ix].cpu().numpy() for p in members])
                H = 16 * m + 256
                ref = orc.Heap(P, H)
                for r in range(P):
                    ref.view(r, 0, m, np.int64)[:] = x[r]
                ref.reduce((0, 1, P), 8 * m, 0, m, W.DT_INT64, W.RED_SUM)
                want = ref.view(0, 8 * m, m, np.int64)
                dt = torch.int64
            elif fmt < 0:
                x = np.stack([wl.heap.view(src, p, torch.float32, n)[ix].cpu().numpy() for p in members])
                ref = orc.Heap(P, 8 * m + 256)
                for r in range(P):
                    ref.view(r, 0, m, np.float32)[:] = x[r]
                ref.reduce((0, 1, P), 4 * m, 0, m, W.DT_FLOAT, W.RED_SUM)
                want = ref.view(0, 4 * m, m, np.float32)
                dt = torch.float32
            else:
                qb = 2 if fmt == 0 else 1
                qt = torch.int16 if fmt == 0 else torch.int8
                qnp = np.int16 if fmt == 0 else np.int8
                nbk = len(blocks)
                bix = torch.from_numpy(blocks).cuda()
                q = np.stack([wl.heap.view(codes, p, qt, n)[ix].cpu().numpy() for p in members])
                s = np.stack([wl.heap.view(sc, p, torch.float32, (n + 127) // 128)[bix].cpu().numpy() for p in members])
                qo, so = 0, (qb * m + 255) // 256 * 256
                do = (so + 4 * nbk + 255) // 256 * 256
                ref = orc.Heap(P, do + 4 * m + 256)
                for r in range(P):
                    ref.view(r, qo, m, qnp)[:] = q[r]
                    ref.view(r, so, nbk, np.float32)[:] = s[r]
                ref.qsum_reduce((0, 1, P), do, qo, so, fmt, m)
                want = ref.view(0, do, m, np.float32)
                dt = torch.float32
            for p in (st0, st0 + P - 1):
                got = wl.heap.view(dst, p, dt, n)[ix].cpu().numpy()
                assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (fmt, t, p)
    finally:
        b.destroy()
