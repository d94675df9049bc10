"""Participation scopes of device-initiated operations (Sec. 6.3): the same script with
a share of its RMA, put_signal, barrier and collective ops flagged warp scope
(SHMEMG_OP_WARP: one warp of the PE performs the op) must leave the oracle's heap
bit-exactly, in every PE mode; the flag is invalid on other kinds."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu

WARP_KINDS = (W.OP_PUT, W.OP_GET, W.OP_PUT_NBI, W.OP_GET_NBI, W.OP_PUT_SIGNAL, W.OP_BARRIER_ALL, W.OP_TEAM_SYNC,
              W.OP_BCAST, W.OP_FCOLLECT, W.OP_ALLTOALL, W.OP_REDUCE)


def _flag_half(ops, seed):
    """Set the warp-scope flag on about half of the eligible ops (seeded)."""
    out = ops.copy()
    pick = (W.cb64_np(seed, np.arange(len(ops), dtype=np.uint64)) & np.uint64(1)).astype(bool)
    elig = np.isin(out["kind"], WARP_KINDS)
    out["kind"][pick & elig] |= W.OP_WARP
    return out, int((pick & elig).sum())


@pytest.mark.parametrize("mode,cd", [(0, 1), (0, 4), (1, 2)])
def test_warp_scope_script_bitexact(sg, heapf, orc, mode, cd):
    s = W.gen_plain_script(seed=777, n_ops=3000)
    h = heapf(s.npes, s.heap_bytes, pe_mode=mode, cluster_dim=cd)
    upload(h, s.heap)
    ops, nflag = _flag_half(s.ops, 99)
    assert nflag > 500
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    fetched = torch.zeros(len(ops), dtype=torch.int64, device="cuda")
    sg.run_script(dev, len(ops), fetched)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(s.npes, s.heap_bytes, s.heap)
    ref.run_script(s.ops)            # the oracle gets the unflagged list: scope has no data effect
    assert first_diff(download(h), ref.mem) is None


def test_warp_scope_shared_team_and_signals(sg, heapf, orc):
    """Warp-scope shared-team collectives of a clustered CTA-mode heap (they take the
    L2 path with the warp barrier), interleaved with PE-scope ones (DSMEM path), and a
    warp-scope put_signal answered by a PE-scope wait."""
    npes, H, cd = 8, 1 << 20, 4
    h = heapf(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=cd)
    init = random_heap(npes, H, 21)
    init.reshape(npes, H)[:, 1000000:1000008] = 0
    upload(h, init)

    def rec(**kw):
        r = np.zeros((), dtype=W.OP_DTYPE)
        r["issuer"] = -1
        for k, v in kw.items():
            r[k] = v
        return r
    ops = [rec(kind=W.OP_REDUCE | W.OP_WARP, dtype=W.DT_INT64, sub=W.RED_SUM, team=1, dst=300000, src=0, n=3000),
           rec(kind=W.OP_REDUCE, dtype=W.DT_INT32, sub=W.RED_MAX, team=1, dst=340000, src=8, n=1001),
           rec(kind=W.OP_BCAST | W.OP_WARP, team=1, pe=2, dst=360000, src=64, n=5000),
           rec(kind=W.OP_FCOLLECT | W.OP_WARP, team=1, dst=380000, src=128, n=2000),
           rec(kind=W.OP_ALLTOALL | W.OP_WARP, team=0, dst=400000, src=256, n=512),
           rec(kind=W.OP_TEAM_SYNC | W.OP_WARP, team=1),
           rec(kind=W.OP_PUT_SIGNAL | W.OP_WARP, sub=W.SIG_ADD, pe=5, issuer=1, dst=500000, src=0, n=4096,
               operand=7, aux=1000000),
           rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_EQ, issuer=5, dst=1000000, operand=7),
           rec(kind=W.OP_GET, pe=5, issuer=5, dst=600000, src=500000, n=4096),
           rec(kind=W.OP_BARRIER_ALL | W.OP_WARP)]
    ops = np.array(ops, dtype=W.OP_DTYPE)
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.run_script(dev, len(ops), None)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    plain = ops.copy()
    plain["kind"] &= 0xFF
    out = []
    teams = [(0, 1, npes)] + [(g * cd, 1, cd) for g in range(npes // cd)]
    for o in plain:                   # shared-team ops once per cluster group
        if o["kind"] in W.COLLECTIVE_KINDS and o["kind"] != W.OP_BARRIER_ALL and o["team"] == 1:
            for g in range(npes // cd):
                e = o.copy()
                e["team"] = 1 + g
                out.append(e)
        else:
            out.append(o)
    ref = orc.Heap(npes, H, init)
    ref.run_script(np.array(out, dtype=W.OP_DTYPE), teams=teams)
    assert first_diff(download(h), ref.mem) is None


def test_warp_flag_rejected_on_amo(sg, heapf):
    npes, H = 2, 1 << 16
    heapf(npes, H)
    ops = np.zeros(2, W.OP_DTYPE)
    ops[0] = (W.OP_BARRIER_ALL, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0)
    ops[1] = (W.OP_FADD | W.OP_WARP, W.DT_INT64, 0, 0, 1, 0, 64, 0, 0, 5, 0, 0)
    sg.clear_status()
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.run_script(dev, 2, None)
    torch.cuda.synchronize()
    code, detail = sg.get_status()
    assert code == sg.ERR_INVALID_ARG and detail == 1
    sg.clear_status()


def test_capabilities_report_warp_scope(sg, heapf):
    heapf(2, 1 << 16)
    caps = sg.query_capabilities(sg.TEAM_WORLD)
    assert caps["coll_scopes"] & 2 and caps["rma_scopes"] & 2      # SHMEMG_SCOPE_WARP
