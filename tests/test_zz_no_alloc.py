"""The allocation-free batched reduce (shmemg_batch_reduce_noalloc) against the
allocating entry point (shmemg_batch_create + shmemg_batch_launch).

Callers that cannot allocate device memory -- a framework whose caching allocator
already holds the GPU, or a loop that must not call cudaMalloc/cudaFree -- use the
allocation-free call; it must give the same outputs as the allocating one, every time
it is called (its scratch array is reused from call to call).  Collected last on
purpose: a run that stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff

pytestmark = pytest.mark.gpu


def _setup(sg, h, world):
    bt = W.gen_batch_teams(seed=5, n_teams=12, world=world, p_hi=world, n_lo=100, n_hi=30000)
    fmts = [-1, 0, 1, -1]
    descs = []
    tmp = h.malloc(4 * 30000)
    for t in range(len(bt.size)):
        n, start, size = int(bt.n[t]), int(bt.start[t]), int(bt.size[t])
        if bt.is_int[t]:
            src, dst = h.malloc(8 * n), h.malloc(8 * n)
            v = W.uniform_ints_np(t, np.arange(world * n, dtype=np.uint64), -(1 << 20), 1 << 20).reshape(world, n)
            for p in range(world):
                h.view(src, p, torch.int64, n).copy_(torch.from_numpy(v[p]))
            descs.append(sg.CollDesc(start, size, sg.INT64, -1, n, dst.ptr, src.ptr, None))
            continue
        fmt = fmts[t % 4]
        x = W.normals_np(300 + t, world * n).astype(np.float32).reshape(world, n)
        dst = h.malloc(4 * n)
        if fmt < 0:
            src = h.malloc(4 * n)
            for p in range(world):
                h.view(src, p, torch.float32, n).copy_(torch.from_numpy(x[p]))
            descs.append(sg.CollDesc(start, size, sg.FLOAT, -1, n, dst.ptr, src.ptr, None))
        else:
            src = h.malloc((2 if fmt == 0 else 1) * n)
            sc = h.malloc(4 * ((n + 127) // 128))
            for p in range(world):
                h.view(tmp, p, torch.float32, n).copy_(torch.from_numpy(x[p]))
            sg.quantize(sg.TEAM_WORLD, src, sc, tmp, fmt, n)
            descs.append(sg.CollDesc(start, size, sg.FLOAT, fmt, n, dst.ptr, src.ptr, sc.ptr))
    torch.cuda.synchronize()
    return descs


def test_noalloc_matches_allocating_entry_point(sg, heapf):
    world, H = 16, 2 << 20
    h = heapf(world, H)
    descs = _setup(sg, h, world)
    init = download(h)
    b = sg.Batch(descs, sg.Tune(2048, 0, 0, 0))
    b.launch()
    torch.cuda.synchronize()
    want = download(h)
    b.destroy()
    assert first_diff(want, init) is not None       # the reduce wrote its outputs
    parts = h.partitions()
    for _ in range(2):                               # two calls in a row, fresh inputs each
        parts.copy_(torch.from_numpy(init.reshape(world, H)).cuda())
        sg.batch_reduce_noalloc(descs, 2048)
        torch.cuda.synchronize()
        assert first_diff(download(h), want) is None
    parts.copy_(torch.from_numpy(init.reshape(world, H)).cuda())
    sg.batch_reduce_noalloc(descs, 2048)             # back to back on one stream
    sg.batch_reduce_noalloc(descs, 2048)
    torch.cuda.synchronize()
    assert first_diff(download(h), want) is None
    assert sg.get_status()[0] == 0


def test_noalloc_rejects_more_than_its_array_holds(sg, heapf):
    world, H = 4, 1 << 20
    h = heapf(world, H)
    src, dst = h.malloc(4 * 16384), h.malloc(4 * 16384)
    d = sg.CollDesc(0, world, sg.FLOAT, -1, 16384, dst.ptr, src.ptr, None)
    with pytest.raises(sg.ShmemgError) as e:           # 600 teams x 128 items > 65536 items
        sg.batch_reduce_noalloc([d] * 600, 128)
    assert e.value.code == sg.ERR_INVALID_ARG
    with pytest.raises(sg.ShmemgError) as e:           # more descriptors than the table holds
        sg.batch_reduce_noalloc([d] * 1025, 16384)
    assert e.value.code == sg.ERR_INVALID_ARG
