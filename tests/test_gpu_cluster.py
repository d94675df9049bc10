"""GPU parity of the cluster-resident shared-team path: device-initiated scripts whose
shared-team barriers are the hardware cluster barrier and whose small shared-team
alltoalls are staged through distributed shared memory (CTA-mode heaps launched in
clusters), and the DSMEM put-with-signal ping-pong.  The oracle runs each shared-team op
once per cluster group, as an explicit team."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20
SRC_INT, SRC_FLT, DST0 = 0, 1 * MiB, 3 * MiB // 2
SHARED = 1


def _rec(**kw):
    r = np.zeros((), dtype=W.OP_DTYPE)
    r["issuer"] = -1
    for k, v in kw.items():
        r[k] = v
    return r


class _Dst:
    """Bump allocator of destination ranges (every op writes a range no other op touches)."""

    def __init__(self, H):
        self.at, self.H = DST0, H

    def take(self, nbytes, skew=0):
        off = (self.at + 255) // 256 * 256 + skew
        self.at = off + nbytes
        assert self.at <= self.H
        return off


def _cluster_script(npes, cd, H):
    """Shared-team reduce / broadcast / fcollect / alltoall / team_sync, alltoalls both
    staged through the DSMEM windows (up to 8 KiB per member) and not, at aligned and
    unaligned offsets, mixed with world ops."""
    d = _Dst(H)
    ops = []
    P = cd
    for dt, op, n, skew in [(W.DT_INT32, W.RED_SUM, 1000, 0), (W.DT_INT64, W.RED_MAX, 777, 8),
                            (W.DT_FLOAT, W.RED_SUM, 4096, 0), (W.DT_FLOAT, W.RED_SUM, 1001, 4),
                            (W.DT_INT32, W.RED_MIN, 40000, 0), (W.DT_FLOAT, W.RED_SUM, 50000, 0),
                            (W.DT_FLOAT, W.RED_MAX, 333, 4), (W.DT_INT64, W.RED_SUM, 16384, 0)]:
        es = 8 if dt == W.DT_INT64 else 4
        src = SRC_FLT + 64 * es if dt == W.DT_FLOAT else SRC_INT + 24 * es
        ops.append(_rec(kind=W.OP_REDUCE, dtype=dt, sub=op, team=SHARED, dst=d.take(n * es, skew), src=src, n=n))
    ops.append(_rec(kind=W.OP_TEAM_SYNC, team=SHARED))
    for n, root in [(5000, P - 1), (200000, 0), (3, P // 2), (128 * KiB, 1)]:
        ops.append(_rec(kind=W.OP_BCAST, team=SHARED, pe=root, dst=d.take(n, 4 if n == 3 else 0), src=SRC_INT + 48, n=n))
    ops.append(_rec(kind=W.OP_PUT, pe=npes - 1, issuer=0, dst=d.take(4096), src=SRC_INT + 8, n=4096))
    ops.append(_rec(kind=W.OP_BARRIER_ALL))
    for n in (3000, 140000, 1 << 17):
        ops.append(_rec(kind=W.OP_FCOLLECT, team=SHARED, dst=d.take(n * P), src=SRC_INT + 16, n=n))
    # (at P = 8: 1024-byte blocks are exactly the 8 KiB per member that is still staged,
    # 1040-byte blocks the first size past it)
    for n in (1000, 20000, 24, 1024, 1040):
        ops.append(_rec(kind=W.OP_ALLTOALL, team=SHARED, dst=d.take(n * P), src=SRC_INT + 32, n=n))
    ops.append(_rec(kind=W.OP_REDUCE, dtype=W.DT_FLOAT, sub=W.RED_SUM, team=0, dst=d.take(4 * 3000), src=SRC_FLT, n=3000))
    ops.append(_rec(kind=W.OP_TEAM_SYNC, team=SHARED))
    return np.array(ops, dtype=W.OP_DTYPE)


def _expand_shared(ops, npes, cd):
    """The oracle's form: each shared-team op once per cluster group (explicit teams
    1 + g = PEs [g*cd, (g+1)*cd))."""
    out = []
    for o in ops:
        if o["kind"] in W.COLLECTIVE_KINDS and o["kind"] != W.OP_BARRIER_ALL and o["team"] == SHARED:
            for g in range(npes // cd):
                e = o.copy()
                e["team"] = 1 + g
                out.append(e)
        else:
            out.append(o)
    teams = [(0, 1, npes)] + [(g * cd, 1, cd) for g in range(npes // cd)]
    return np.array(out, dtype=W.OP_DTYPE), teams


def _init_heap(npes, H, seed):
    init = random_heap(npes, H, seed)
    m = init.reshape(npes, H)
    m[:, SRC_FLT:SRC_FLT + 256 * KiB] = W.normals_np(seed + 1, npes * 64 * KiB).astype(np.float32) \
        .view(np.uint8).reshape(npes, 256 * KiB)
    return init


def test_shared_team_path_reports_dsmem(sg, heapf):
    heapf(8, 1 << 16, pe_mode=sg.PE_MODE_CTA, cluster_dim=4)
    assert sg.query_capabilities(sg.TEAM_SHARED)["path"] & 2
    assert sg.query_capabilities(sg.TEAM_WORLD)["path"] == 1


@pytest.mark.parametrize("cd", [2, 4, 8])
def test_cluster_shared_script_bitexact(sg, heapf, orc, cd):
    npes, H = 16, 8 * MiB
    h = heapf(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=cd)
    init = _init_heap(npes, H, 100 + cd)
    upload(h, init)
    ops = _cluster_script(npes, cd, H)
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.clear_status()
    sg.run_script(dev, len(ops), None)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(npes, H, init)
    eops, teams = _expand_shared(ops, npes, cd)
    ref.run_script(eops, teams=teams)
    assert first_diff(download(h), ref.mem) is None


def test_cluster_script_repeated_launches(sg, heapf, orc):
    """Many shared-team barriers, reductions and staged alltoalls in one launch and
    across launches (barrier generations start afresh in every launch)."""
    npes, H, cd = 8, 4 * MiB, 4
    h = heapf(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=cd)
    init = _init_heap(npes, H, 7)
    upload(h, init)
    ops = []
    for k in range(200):
        ops.append(_rec(kind=W.OP_REDUCE, dtype=W.DT_INT64, sub=W.RED_SUM, team=SHARED,
                        dst=DST0 + (k % 50) * 4096, src=SRC_INT + 8 * k, n=64 + k))
        ops.append(_rec(kind=W.OP_TEAM_SYNC, team=SHARED))
        ops.append(_rec(kind=W.OP_ALLTOALL, team=SHARED, dst=2 * MiB + (k % 50) * 4096, src=SRC_INT + 16 * k,
                        n=16 + (k % 8) * 16))
    ops = np.array(ops, dtype=W.OP_DTYPE)
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    ref = orc.Heap(npes, H, init)
    eops, teams = _expand_shared(ops, npes, cd)
    for _ in range(3):
        sg.run_script(dev, len(ops), None)
        ref.run_script(eops, teams=teams)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    assert first_diff(download(h), ref.mem) is None


@pytest.mark.parametrize("cd", [2, 4])
@pytest.mark.parametrize("payload", [8, 1000, 4096])
def test_pingpong_cluster_final_state(sg, heapf, orc, cd, payload):
    npairs, iters, npes = 16, 200, 32
    H = 3 * 4096 + 256
    h = heapf(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=cd)
    init = random_heap(npes, H, payload + cd)
    init.reshape(npes, H)[:, 3 * 4096:3 * 4096 + 8] = 0
    upload(h, init)
    lat = torch.zeros(npairs * iters, dtype=torch.int64, device="cuda")
    sg.pingpong_cluster(h.base, h.base + 3 * 4096, payload, npairs, iters, lat)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(npes, H, init)
    for k in range(npairs):
        a, b = 2 * k, 2 * k + 1
        for _ in range(iters):
            ref.put_signal(payload, 0, payload, 3 * 4096, W.SIG_ADD, 1, b, a)
            ref.put_signal(payload, 0, payload, 3 * 4096, W.SIG_ADD, 1, a, b)
    assert first_diff(download(h), ref.mem) is None
    assert bool((lat > 0).all())


def test_pingpong_cluster_zero_rounds_keeps_heap(sg, heapf):
    npes, H = 4, 8192
    h = heapf(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=2)
    init = random_heap(npes, H, 3)
    upload(h, init)
    sg.pingpong_cluster(h.base, h.base + 4096, 512, 2, 0, None)
    assert first_diff(download(h), init) is None


def test_pingpong_cluster_needs_cluster_heap(sg, heapf):
    h = heapf(4, 8192)
    with pytest.raises(sg.ShmemgError) as e:
        sg.pingpong_cluster(h.base, h.base + 4096, 64, 2, 1, None)
    assert e.value.code == sg.ERR_UNSUPPORTED


def test_cluster_barrier_timeout_is_bounded(sg, heapf):
    """PE 1 waits on a signal nobody raises and times out; having failed, it still
    passes the shared-team (cluster) barrier of the next op, where PE 0 waits for it, so
    the launch ends; the status names the timeout and the context survives."""
    npes, H = 2, 4096
    h = heapf(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=2, timeout_ns=3_000_000)
    h.partitions().zero_()
    ops = np.zeros(2, W.OP_DTYPE)
    ops[0] = (W.OP_WAIT_UNTIL, 0, W.CMP_EQ, 0, 0, 1, 0, 0, 0, 12345, 0, 0)
    ops[1] = (W.OP_TEAM_SYNC, 0, 0, SHARED, 0, -1, 0, 0, 0, 0, 0, 0)
    sg.clear_status()
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.run_script(dev, 2, None)
    torch.cuda.synchronize()
    code, detail = sg.get_status()
    assert code == sg.ERR_TIMEOUT and detail == 0
    sg.clear_status()
    x = torch.ones(4, device="cuda")
    assert float(x.sum()) == 4.0


def test_cluster_failed_pe_keeps_barrier_sequence(sg, heapf):
    """After PE 1 fails (a timed-out wait), the ops that follow -- shared-team syncs,
    staged and unstaged shared-team collectives, a world barrier -- still end: the failed
    PE walks the rest of the script through each op's cluster barriers, the others learn
    of the failure at the world barrier, and the launch returns with the timeout
    recorded."""
    npes, H, cd = 8, 1 << 20, 4
    h = heapf(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=cd, timeout_ns=3_000_000)
    h.partitions().zero_()
    ops = [_rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_EQ, issuer=1, dst=0, operand=12345),
           _rec(kind=W.OP_TEAM_SYNC, team=SHARED),
           _rec(kind=W.OP_REDUCE, dtype=W.DT_INT64, sub=W.RED_SUM, team=SHARED, dst=65536, src=4096, n=1000),
           _rec(kind=W.OP_REDUCE, dtype=W.DT_INT32, sub=W.RED_MAX, team=SHARED, dst=131072, src=4096, n=60000),
           _rec(kind=W.OP_BCAST, team=SHARED, pe=2, dst=524288, src=4096, n=3000),
           _rec(kind=W.OP_BARRIER_ALL),
           _rec(kind=W.OP_ALLTOALL, team=SHARED, dst=600000, src=4096, n=64),
           _rec(kind=W.OP_ALLTOALL, team=SHARED, dst=700000, src=4096, n=4096),
           _rec(kind=W.OP_TEAM_SYNC, team=SHARED)]
    ops = np.array(ops, dtype=W.OP_DTYPE)
    sg.clear_status()
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.run_script(dev, len(ops), None)
    torch.cuda.synchronize()
    code, detail = sg.get_status()
    assert code == sg.ERR_TIMEOUT and detail == 0
    sg.clear_status()
    assert float(torch.ones(4, device="cuda").sum()) == 4.0
