"""Full-size parity of the halo-exchange workload as the benchmark times it: 19 x 8 PEs
(one per SM) of 1024 x 1024 binary32 tiles, 100 Jacobi sweeps, persistent (PE = one CTA
and PE = a 2-CTA cluster) and launch-per-sweep.  After T sweeps a point depends only on
the points within distance T of it, so the oracle runs the T sweeps on the (2T+3)-square
window of the initial grid centred on a sampled point (periodic wrap inside the window
cannot reach the centre) and its centre must equal the GPU's value bitwise.  Samples:
tile corners and edges (where the halos feed in) and random points.  The three GPU runs
must also agree with each other on the whole grid."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

PX, PY, NX, NY, T = 19, 8, 1024, 1024, 100
NPES = PX * PY


def _points():
    pts = []
    for p in (0, 7, 93, NPES - 1):   # corners and edge midpoints of a few tiles
        x, y = p % PX, p // PX
        for i, j in ((0, 0), (0, NX - 1), (NY - 1, 0), (NY - 1, NX - 1), (0, NX // 2), (NY // 2, 0),
                     (NY - 1, 3), (5, NX - 1)):
            pts.append((y * NY + i, x * NX + j))
    r = W.cb64_np(W.derive_seed("halo-points"), np.arange(16, dtype=np.uint64))
    for k in range(16):
        pts.append((int(r[k] % np.uint64(PY * NY)), int((r[k] >> np.uint64(32)) % np.uint64(PX * NX))))
    return pts


def _run(sg, mode, cd, init, plain):
    hs = sg.halo_stride(NX, NY)
    tile_b, halo_b = 2 * NX * NY * 4, 2 * hs * 4
    heap = sg.Heap(NPES, (tile_b + halo_b + 64 + 4095) // 4096 * 4096, pe_mode=mode, cluster_dim=cd)
    try:
        parts = heap.partitions()
        parts.zero_()
        parts[:, :NX * NY * 4].view(torch.float32).copy_(init)
        sg.clear_status()
        sg.halo_jacobi(heap.sym(0, tile_b), heap.sym(tile_b, halo_b), heap.sym(tile_b + halo_b, 32), PX, PY, NX, NY,
                       T, plain=plain)
        torch.cuda.synchronize()
        assert sg.get_status()[0] == 0
        r0 = (T & 1) * NX * NY * 4
        return parts[:, r0:r0 + NX * NY * 4].view(torch.float32).clone()
    finally:
        heap.close()


def test_halo_full_size_light_cones(sg, orc):
    torch.cuda.set_device(0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(W.derive_seed("halo") & 0x7FFFFFFF)
    init = torch.randn(NPES, NX * NY, device="cuda", generator=gen)
    got = _run(sg, sg.PE_MODE_CTA, 1, init, plain=False)
    assert torch.equal(_run(sg, sg.PE_MODE_CLUSTER, 2, init, plain=False), got)
    assert torch.equal(_run(sg, sg.PE_MODE_CTA, 1, init, plain=True), got)
    tiles = init.cpu().numpy().reshape(PY, PX, NY, NX)
    grid = tiles.transpose(0, 2, 1, 3).reshape(PY * NY, PX * NX)   # global row-major grid
    out = got.cpu().numpy().reshape(PY, PX, NY, NX).transpose(0, 2, 1, 3).reshape(PY * NY, PX * NX)
    d = np.arange(-(T + 1), T + 2)
    for gy, gx in _points():
        win = grid[np.ix_((gy + d) % grid.shape[0], (gx + d) % grid.shape[1])]
        want = orc.halo_jacobi(win, T)[T + 1, T + 1]
        assert np.float32(out[gy, gx]).view(np.uint32) == np.float32(want).view(np.uint32), (gy, gx)
