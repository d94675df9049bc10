"""GPU parity of the integer reductions that take the bulk ring (k_reduce_bulk: teams of
48..64 members with at least 128 KiB per member, 1 KiB per member per chunk, three
stages): the smallest team and size that take it, ragged last chunks down to one vector,
rings that wrap many times, strided teams, in place, and the neighbours that do not take it
(47 and 65 members, 16 bytes under the threshold); bit-exact heaps against the oracle
(paper Sec. 6.3 reductions: every member receives the combination of all members)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu

KiB = 1 << 10


def _ops(sg):
    return [(sg.INT32, 4, sg.SUM), (sg.INT32, 4, sg.MAX), (sg.INT64, 8, sg.MIN), (sg.INT64, 8, sg.SUM)]


def _heap(npes, member_bytes):
    H = 2 * member_bytes + 64 * KiB
    return (H + 255) // 256 * 256, (member_bytes + 32 * KiB + 255) // 256 * 256


@pytest.mark.parametrize("npes,member_bytes", [(48, 128 * KiB), (64, 256 * KiB + 48), (64, 2 * 1024 * KiB + 32),
                                               (57, 1024 * KiB + 1040), (64, 128 * KiB - 16), (47, 256 * KiB),
                                               (65, 256 * KiB + 16)])
def test_bulk_ring_world(sg, heapf, orc, npes, member_bytes):
    H, dst = _heap(npes, member_bytes)
    h = heapf(npes, H)
    init = random_heap(npes, H, npes * 7 + member_bytes)
    upload(h, init)
    ref = orc.Heap(npes, H, init)
    for dt, es, op in _ops(sg):
        n = member_bytes // es
        sg.reduce(sg.TEAM_WORLD, h.base + dst, h.base + 0, n, dt, op)
        ref.reduce((0, 1, npes), dst, 0, n, dt, op)
    # in place, last
    sg.reduce(sg.TEAM_WORLD, h.base + 0, h.base + 0, member_bytes // 8, sg.INT64, sg.SUM)
    ref.reduce((0, 1, npes), 0, 0, member_bytes // 8, W.DT_INT64, W.RED_SUM)
    got = download(h)
    assert first_diff(got, ref.mem) is None, first_diff(got, ref.mem)


def test_bulk_ring_strided_teams(sg, heapf, orc):
    npes, member_bytes = 130, 512 * KiB + 64
    H, dst = _heap(npes, member_bytes)
    h = heapf(npes, H)
    init = random_heap(npes, H, 4401)
    upload(h, init)
    ref = orc.Heap(npes, H, init)
    for start, stride, size in [(1, 2, 64), (0, 1, 48), (7, 2, 50)]:
        t = sg.team_split_strided(sg.TEAM_WORLD, start, stride, size)
        for dt, es, op in _ops(sg):
            n = member_bytes // es
            sg.reduce(t, h.base + dst, h.base + 0, n, dt, op)
            ref.reduce((start, stride, size), dst, 0, n, dt, op)
        sg.team_destroy(t)
    got = download(h)
    assert first_diff(got, ref.mem) is None, first_diff(got, ref.mem)
