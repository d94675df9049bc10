"""Explicit device contexts (Sec. 6.2): non-blocking puts and gets on contexts 1..3 move
in the background and complete at quiet on their context (or on all); the final heap
equals the oracle's (which applies every op at once) whenever the script quiets before it
reads, in every PE mode; the queue, the kernel's end and invalid contexts are covered."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu
KiB, MiB = 1 << 10, 1 << 20
ALL = 0xFF


def _rec(**kw):
    r = np.zeros((), dtype=W.OP_DTYPE)
    r["issuer"] = -1
    for k, v in kw.items():
        r[k] = v
    return r


def _run(sg, h, orc, init, ops):
    ops = np.array(ops, dtype=W.OP_DTYPE)
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.clear_status()
    sg.run_script(dev, len(ops), None)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(h.npes, h.H, init)
    ref.run_script(ops)
    return first_diff(download(h), ref.mem)


@pytest.mark.parametrize("mode,cd", [(0, 1), (0, 2), (1, 2)])
def test_context_transfers_bitexact(sg, heapf, orc, mode, cd):
    npes, H = 8, 8 * MiB
    h = heapf(npes, H, pe_mode=mode, cluster_dim=cd)
    init = random_heap(npes, H, 30 + mode)
    upload(h, init)
    ops = []
    for p in range(npes):
        ops += [_rec(kind=W.OP_PUT_NBI, sub=1, pe=(p + 1) % npes, issuer=p, dst=2 * MiB, src=0, n=MiB + 48),
                _rec(kind=W.OP_GET_NBI, sub=2, pe=(p + 2) % npes, issuer=p, dst=4 * MiB, src=MiB + 512, n=300 * KiB),
                _rec(kind=W.OP_PUT_NBI, sub=3, pe=(p + 3) % npes, issuer=p, dst=5 * MiB + 8, src=8, n=1000),  # unaligned
                _rec(kind=W.OP_PUT, pe=(p + 5) % npes, issuer=p, dst=6 * MiB + 4096 * p, src=64, n=4096)]
    for p in range(npes):
        ops += [_rec(kind=W.OP_QUIET, sub=1, issuer=p), _rec(kind=W.OP_QUIET, sub=2, issuer=p),
                _rec(kind=W.OP_QUIET, sub=ALL, issuer=p)]
    ops += [_rec(kind=W.OP_BARRIER_ALL)]
    for p in range(npes):   # read what the contexts delivered
        ops += [_rec(kind=W.OP_GET, pe=(p + 1) % npes, issuer=p, dst=7 * MiB, src=2 * MiB + 4096, n=64 * KiB)]
    assert _run(sg, h, orc, init, ops) is None


def test_context_queue_overflow_and_end_of_script(sg, heapf, orc):
    """More transfers than a context queues (its queue drains to make room), and
    transfers never quieted (the script's end completes them)."""
    npes, H = 4, 4 * MiB
    h = heapf(npes, H)
    init = random_heap(npes, H, 41)
    upload(h, init)
    ops = []
    for k in range(20):   # PE 0 queues 14 transfers on context 1 (8 fit), the rest on context 2
        ops.append(_rec(kind=W.OP_PUT_NBI, sub=1 if k < 14 else 2, pe=1 + k % 3, issuer=0,
                        dst=2 * MiB + 32 * KiB * k, src=16 * KiB * k, n=32 * KiB))
    assert _run(sg, h, orc, init, ops) is None


def test_context_overlaps_default_context_work(sg, heapf, orc):
    """A large transfer on context 1 while the same PEs run blocking puts and
    put_signal / wait pairs on the default context; only then quiet context 1."""
    npes, H = 4, 32 * MiB
    h = heapf(npes, H)
    init = random_heap(npes, H, 52)
    init.reshape(npes, H)[:, 31 * MiB:31 * MiB + 64] = 0
    upload(h, init)
    ops = [_rec(kind=W.OP_PUT_NBI, sub=1, pe=(p + 1) % npes, issuer=p, dst=16 * MiB, src=0, n=12 * MiB)
           for p in range(npes)]
    for k in range(50):
        p = k % npes
        ops.append(_rec(kind=W.OP_PUT, pe=(p + 2) % npes, issuer=p, dst=30 * MiB + 4096 * k, src=13 * MiB, n=4096))
    ops.append(_rec(kind=W.OP_PUT_SIGNAL, sub=W.SIG_ADD, pe=1, issuer=0, dst=29 * MiB, src=14 * MiB, n=8192,
                    operand=1, aux=31 * MiB))
    ops.append(_rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_GE, issuer=1, dst=31 * MiB, operand=1))
    ops += [_rec(kind=W.OP_QUIET, sub=1, issuer=p) for p in range(npes)]
    ops.append(_rec(kind=W.OP_BARRIER_ALL))
    assert _run(sg, h, orc, init, ops) is None


@pytest.mark.parametrize("mode,cd", [(0, 1), (1, 2)])
def test_blocking_bulk_copies_behind_context_chunks(sg, heapf, orc, mode, cd):
    """Large blocking puts and gets (the bulk engine's queue 0) issued while context
    transfers are still in the ring: they join the queue behind the chunks in flight and
    still complete before the op returns (the get reads what the put wrote)."""
    npes, H = 4, 32 * MiB
    h = heapf(npes, H, pe_mode=mode, cluster_dim=cd)
    init = random_heap(npes, H, 63 + mode)
    upload(h, init)
    ops = []
    for p in range(npes):
        ops += [_rec(kind=W.OP_PUT_NBI, sub=1, pe=(p + 1) % npes, issuer=p, dst=16 * MiB, src=0, n=10 * MiB),
                _rec(kind=W.OP_GET_NBI, sub=3, pe=(p + 3) % npes, issuer=p, dst=27 * MiB, src=MiB, n=2 * MiB)]
    for p in range(npes):   # blocking bulk copies while the contexts' chunks are in flight
        ops += [_rec(kind=W.OP_PUT, pe=(p + 2) % npes, issuer=p, dst=12 * MiB + MiB * p, src=11 * MiB, n=MiB),
                _rec(kind=W.OP_GET, pe=(p + 2) % npes, issuer=p, dst=30 * MiB, src=12 * MiB + MiB * p, n=MiB)]
    ops += [_rec(kind=W.OP_QUIET, sub=ALL, issuer=p) for p in range(npes)]
    ops.append(_rec(kind=W.OP_BARRIER_ALL))
    assert _run(sg, h, orc, init, ops) is None


def test_context_chunks_drain_before_a_staged_cluster_alltoall(sg, heapf, orc):
    """CTA PEs in clusters of 4: context transfers in flight when a shared-team alltoall
    stages its blocks in the same shared-memory ring (its DSMEM window); the ring drains
    first, and the transfers, the staged alltoall and the collectives after it (through
    L2 between cluster barriers) come out right."""
    npes, H = 8, 8 * MiB
    h = heapf(npes, H, pe_mode=0, cluster_dim=4)
    init = random_heap(npes, H, 71)
    upload(h, init)
    ops = []
    for p in range(npes):
        ops.append(_rec(kind=W.OP_PUT_NBI, sub=2, pe=(p + 4) % npes, issuer=p, dst=4 * MiB, src=0, n=3 * MiB))
    ops += [_rec(kind=W.OP_ALLTOALL, team=1, dst=7 * MiB + 262144, src=3 * MiB + 32768, n=1024),
            _rec(kind=W.OP_REDUCE, dtype=W.DT_INT64, sub=W.RED_SUM, team=1, dst=7 * MiB, src=3 * MiB + 4096, n=2048),
            _rec(kind=W.OP_BCAST, team=1, pe=2, dst=7 * MiB + 65536, src=3 * MiB, n=8192),
            _rec(kind=W.OP_FCOLLECT, team=1, dst=7 * MiB + 131072, src=3 * MiB + 16384, n=4096)]
    ops += [_rec(kind=W.OP_QUIET, sub=2, issuer=p) for p in range(npes)]
    ops.append(_rec(kind=W.OP_BARRIER_ALL))
    ops = np.array(ops, dtype=W.OP_DTYPE)
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.clear_status()
    sg.run_script(dev, len(ops), None)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    # the oracle's form: each shared-team op once per cluster (explicit teams 1 + g)
    eops = []
    for o in ops:
        if o["kind"] in W.COLLECTIVE_KINDS and o["kind"] != W.OP_BARRIER_ALL and o["team"] == 1:
            for g in range(npes // 4):
                e = o.copy()
                e["team"] = 1 + g
                eops.append(e)
        else:
            eops.append(o)
    ref = orc.Heap(npes, H, init)
    ref.run_script(np.array(eops, dtype=W.OP_DTYPE), teams=[(0, 1, npes)] + [(4 * g, 1, 4) for g in range(npes // 4)])
    assert first_diff(download(h), ref.mem) is None


@pytest.mark.parametrize("bad", [
    dict(kind=W.OP_PUT_NBI, sub=4, pe=1, issuer=0, dst=0, src=4096, n=64),     # no context 4
    dict(kind=W.OP_QUIET, sub=7, issuer=0),                                     # no context 7
    dict(kind=W.OP_PUT_NBI | W.OP_WARP, sub=1, pe=1, issuer=0, dst=0, src=4096, n=64)])  # warp scope on a context
def test_invalid_contexts_rejected(sg, heapf, bad):
    h = heapf(2, 1 << 16)
    ops = np.array([_rec(kind=W.OP_BARRIER_ALL), _rec(**bad)], dtype=W.OP_DTYPE)
    sg.clear_status()
    sg.run_script(torch.from_numpy(ops.view(np.uint8).copy()).cuda(), 2, None)
    torch.cuda.synchronize()
    code, detail = sg.get_status()
    assert code == sg.ERR_INVALID_ARG and detail == 1
    sg.clear_status()


@pytest.mark.parametrize("npes", [96, 6])
def test_contexts_with_and_without_agents(sg, heapf, orc, npes):
    """CTA PEs without clusters: 6 PEs get a context agent each (a second CTA), 96 PEs do
    not fit twice on the GPU and keep their contexts on their own engine.  Both: three
    contexts per PE with transfers interleaved with blocking puts, a quiet on one context
    while the others still move (context independence), a get of what a quieted context
    delivered, and transfers left for the script's end."""
    H = 4 * MiB
    h = heapf(npes, H)
    init = random_heap(npes, H, 90 + npes)
    upload(h, init)
    ops = []
    for p in range(npes):
        ops += [_rec(kind=W.OP_PUT_NBI, sub=1, pe=(p + 1) % npes, issuer=p, dst=2 * MiB, src=0, n=768 * KiB),
                _rec(kind=W.OP_GET_NBI, sub=2, pe=(p + 2) % npes, issuer=p, dst=3 * MiB, src=256 * KiB, n=256 * KiB),
                _rec(kind=W.OP_PUT, pe=(p + 3) % npes, issuer=p, dst=3 * MiB + 512 * KiB + 64 * p, src=64, n=64),
                _rec(kind=W.OP_PUT_NBI, sub=3, pe=(p + 1) % npes, issuer=p, dst=3 * MiB + 768 * KiB, src=512 * KiB,
                     n=128 * KiB + 16)]
    for p in range(npes):
        ops.append(_rec(kind=W.OP_QUIET, sub=2, issuer=p))
    ops.append(_rec(kind=W.OP_BARRIER_ALL))
    for p in range(npes):   # what context 2 delivered, read back after its quiet and a barrier
        ops.append(_rec(kind=W.OP_GET, pe=(p + 1) % npes, issuer=p, dst=3 * MiB + 640 * KiB, src=3 * MiB, n=64 * KiB))
    assert _run(sg, h, orc, init, ops) is None


def test_context_agents_across_graph_replays(sg, heapf, orc):
    """A script with context transfers captured once in a CUDA graph and replayed: each
    replay adds to a word, moves the block holding it on context 1, quiets, and reads the
    neighbour's copy back; after three replays the heap equals three runs of the oracle
    (every replay's quiet waited for that replay's transfer)."""
    npes, H = 6, 2 * MiB
    h = heapf(npes, H)
    init = random_heap(npes, H, 101)
    upload(h, init)
    W0, D, E = 0, 512 * KiB, 1 * MiB
    ops = []
    for p in range(npes):
        ops += [_rec(kind=W.OP_FADD, dtype=W.DT_INT64, pe=p, issuer=p, dst=W0, operand=1 + p),
                _rec(kind=W.OP_PUT_NBI, sub=1, pe=(p + 1) % npes, issuer=p, dst=D, src=W0, n=256 * KiB),
                _rec(kind=W.OP_QUIET, sub=1, issuer=p)]
    ops.append(_rec(kind=W.OP_BARRIER_ALL))
    for p in range(npes):
        ops.append(_rec(kind=W.OP_GET, pe=(p + 1) % npes, issuer=p, dst=E, src=D, n=64 * KiB))
    ops.append(_rec(kind=W.OP_BARRIER_ALL))
    ops = np.array(ops, dtype=W.OP_DTYPE)
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.clear_status()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sg.run_script(dev, len(ops), None, s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(npes, H, init)
    for _ in range(3):
        ref.run_script(ops)
    assert first_diff(download(h), ref.mem) is None


def test_context_transfer_as_each_pes_last_op(sg, heapf, orc):
    """Each PE's last op is a context transfer with no quiet, barrier or later op: the
    script's end alone must complete it (the PE leaves right after posting it to its
    agent, which must still take it).  Repeated with new data, so a transfer the agent
    missed would leave a stale destination."""
    npes, H = 6, 1 * MiB
    h = heapf(npes, H)
    for it in range(12):
        init = random_heap(npes, H, 500 + it)
        upload(h, init)
        ops = [_rec(kind=W.OP_PUT, pe=(p + 2) % npes, issuer=p, dst=768 * KiB, src=0, n=4096) for p in range(npes)]
        ops += [_rec(kind=W.OP_PUT_NBI, sub=1 + p % 3, pe=(p + 1) % npes, issuer=p, dst=256 * KiB, src=0,
                     n=64 * KiB + 16 * it) for p in range(npes)]
        assert _run(sg, h, orc, init, ops) is None, it
