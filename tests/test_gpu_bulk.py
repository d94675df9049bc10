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
