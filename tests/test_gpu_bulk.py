"""Large device-initiated puts and gets through the bulk (TMA) engine: a ring of
concurrent put_nbi over every PE, a barrier, then a ring of blocking gets of what the
puts wrote; sizes that are and are not multiples of the 32 KiB chunk; both PE modes.
The final heap must equal the oracle's bit for bit."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu

MiB = 1 << 20


@pytest.mark.parametrize("mode,cd", [(0, 1), (1, 2), (1, 4)])
@pytest.mark.parametrize("m", [64 << 10, 3 * MiB + 16, 8 * MiB])
def test_bulk_ring_put_get(sg, heapf, orc, mode, cd, m):
    npes, H = 8, 28 * MiB
    A, B, C = 0, 9 * MiB, 18 * MiB
    h = heapf(npes, H, pe_mode=mode, cluster_dim=cd)
    init = random_heap(npes, H, m + cd)
    upload(h, init)
    ops = []
    for p in range(npes):        # PE p: its A -> B of p+1
        ops.append((W.OP_PUT_NBI, 0, 0, 0, (p + 1) % npes, p, B, A, m, 0, 0, 0))
    ops.append((W.OP_BARRIER_ALL, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0))
    for p in range(npes):        # PE p: B of p+2 -> its C
        ops.append((W.OP_GET, 0, 0, 0, (p + 2) % npes, p, C, B, m, 0, 0, 0))
    ops.append((W.OP_BARRIER_ALL, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0))
    ops = np.array(ops, dtype=W.OP_DTYPE)
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.run_script(dev, len(ops), None)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(npes, H, init)
    ref.run_script(ops)
    d = first_diff(download(h), ref.mem)
    assert d is None, d


def test_bulk_host_collectives(sg, heapf, orc):
    """Host-issued broadcast / fcollect / alltoall / put large enough for the bulk engine
    (ragged last chunk, strided team, per-cluster SHARED groups) against the oracle."""
    npes, H = 8, 4 * MiB
    h = heapf(npes, H, pe_mode=0, cluster_dim=4)
    init = random_heap(npes, H, 77)
    upload(h, init)
    ref = orc.Heap(npes, H, init)
    b = h.base
    sg.broadcastmem(sg.TEAM_WORLD, b + 2 * MiB, b + 0, 100 * 1024 + 16, 5)
    ref.broadcast((0, 1, npes), 2 * MiB, 0, 100 * 1024 + 16, 5)
    t = sg.team_split_strided(sg.TEAM_WORLD, 1, 2, 4)       # PEs 1, 3, 5, 7
    sg.fcollectmem(t, b + 3 * MiB, b + 160 * 1024, 48 * 1024)
    ref.fcollect((1, 2, 4), 3 * MiB, 160 * 1024, 48 * 1024)
    sg.alltoallmem(t, b + 512 * 1024, b + 1024 * 1024, 40 * 1024)
    ref.alltoall((1, 2, 4), 512 * 1024, 1024 * 1024, 40 * 1024)
    sg.team_destroy(t)
    sg.broadcastmem(sg.TEAM_SHARED, b + 1536 * 1024, b + 1024 * 1024, 64 * 1024, 2)
    for g in range(2):
        ref.broadcast((4 * g, 1, 4), 1536 * 1024, 1024 * 1024, 64 * 1024, 2)
    sg.putmem(b + 3584 * 1024, b + 0, 512 * 1024 - 32, 6, 1)
    ref.put(3584 * 1024, 0, 512 * 1024 - 32, 6, 1)
    sg.quiet()
    d = first_diff(download(h), ref.mem)
    assert d is None, d
