"""GPU parity of the halo-exchange workload (paper Sec. 4.4, case study 1): the grid
decomposed into px x py tiles with device-initiated halo puts + signals (one launch)
and with one launch per sweep, each against the oracle's Jacobi on the whole grid,
bit-exactly."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _run(sg, heapf, orc, px, py, nx, ny, iters, mode=0, cd=1, plain=False, seed=3, repeat=1):
    npes = px * py
    hs = sg.halo_stride(nx, ny)
    tile_b, halo_b = 2 * nx * ny * 4, 2 * hs * 4
    H = (tile_b + halo_b + 64 + 4095) // 4096 * 4096
    h = heapf(npes, H, pe_mode=mode, cluster_dim=cd)
    tiles, halos, sigs = h.sym(0, tile_b), h.sym(tile_b, halo_b), h.sym(tile_b + halo_b, 32)
    grid = W.normals_np(seed, npes * nx * ny).astype(np.float32).reshape(py * ny, px * nx)
    parts = h.partitions()
    parts.zero_()
    for p in range(npes):
        x, y = p % px, p // px
        t0 = np.ascontiguousarray(grid[y * ny:(y + 1) * ny, x * nx:(x + 1) * nx])
        h.view(tiles, p, torch.float32, nx * ny).copy_(torch.from_numpy(t0.reshape(-1)))
    torch.cuda.synchronize()
    for _ in range(repeat):
        sg.halo_jacobi(tiles, halos, sigs, px, py, nx, ny, iters, plain=plain)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    want = orc.halo_jacobi(grid, iters * repeat)
    res = (iters & 1) * nx * ny * 4
    got = np.zeros_like(grid)
    for p in range(npes):
        x, y = p % px, p // px
        got[y * ny:(y + 1) * ny, x * nx:(x + 1) * nx] = \
            h.view(h.sym(res, nx * ny * 4), p, torch.float32, nx * ny).cpu().numpy().reshape(ny, nx)
    sig = parts[:, tiles.nbytes + halos.nbytes:tiles.nbytes + halos.nbytes + 32].cpu().numpy()
    return got, want, sig


@pytest.mark.parametrize("plain", [False, True])
@pytest.mark.parametrize("px,py,nx,ny,iters", [(4, 2, 64, 48, 7), (1, 1, 16, 8, 5), (2, 1, 32, 5, 4),
                                                (3, 2, 40, 7, 9), (2, 3, 4, 1, 3), (4, 4, 2048, 16, 2),
                                                (2, 2, 2208, 9, 3), (3, 1, 384, 37, 5)])
def test_halo_jacobi_matches_whole_grid(sg, heapf, orc, px, py, nx, ny, iters, plain):
    got, want, sig = _run(sg, heapf, orc, px, py, nx, ny, iters, plain=plain)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert not sig.any()                      # signals left zero for the next run


@pytest.mark.parametrize("mode,cd", [(0, 2), (1, 2), (1, 4)])
def test_halo_jacobi_pe_modes(sg, heapf, orc, mode, cd):
    got, want, _ = _run(sg, heapf, orc, 4, 2, 256, 33, 6, mode=mode, cd=cd)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_halo_jacobi_repeated_runs(sg, heapf, orc):
    got, want, sig = _run(sg, heapf, orc, 2, 2, 32, 16, 4, repeat=3)   # even iters: result back in tile 0
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)) and not sig.any()


def test_halo_jacobi_zero_iters(sg, heapf, orc):
    got, want, _ = _run(sg, heapf, orc, 2, 2, 32, 16, 0)
    assert np.array_equal(got, want)


def test_halo_jacobi_argument_checks(sg, heapf):
    h = heapf(4, 1 << 16)
    t, hl, s = h.sym(0, 8192), h.sym(16384, 4096), h.sym(32768, 32)
    for args in ((4, 2, 16, 8), (2, 2, 6, 8), (2, 2, 0, 8), (2, 2, 16, 0)):
        with pytest.raises(sg.ShmemgError) as e:
            sg.halo_jacobi(t, hl, s, *args, 1)
        assert e.value.code == sg.ERR_INVALID_ARG
