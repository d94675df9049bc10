"""Conformance tests in the shape the paper lists them (Sec. 8, "Conformance and
Implementation Mapping"): context visibility, space symmetry, the GPU space at
initialisation, ordering/completion (quiet and fence), stream ordering with its
documented constraints (Sec. 6.4: no deadlock with waits in one stream; host and device
collectives on one team only with explicit ordering), pointer accessibility and
progress.  Every check compares against the oracle or a closed form."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu
KiB = 1 << 10


def _rec(**kw):
    r = np.zeros((), dtype=W.OP_DTYPE)
    r["issuer"] = -1
    for k, v in kw.items():
        r[k] = v
    return r


def _dev(ops):
    ops = np.array(ops, dtype=W.OP_DTYPE)
    return ops, torch.from_numpy(ops.view(np.uint8).copy()).cuda()


def test_context_visibility(sg, heapf, orc):
    """A default device context is reported and usable from device code, and so are the
    explicit contexts the capability reports (Sec. 6.2)."""
    npes, H = 4, 1 << 16
    h = heapf(npes, H)
    caps = sg.query_capabilities(sg.TEAM_WORLD)
    assert "DEVICE_CTX_DEFAULT" in caps["flag_names"] and "EXPLICIT_DEVICE_CTX" in caps["flag_names"]
    assert caps["device_ctx_count"] > 1
    ctx = sg.device_ctx()
    assert ctx.npes == npes and ctx.pe_stride == H
    init = random_heap(npes, H, 1)
    upload(h, init)
    ops, dev = _dev([_rec(kind=W.OP_PUT, pe=3, issuer=0, dst=8192, src=0, n=1000),     # default context
                     _rec(kind=W.OP_PUT_NBI, sub=caps["device_ctx_count"] - 1, pe=2, issuer=1, dst=16384, src=0,
                          n=4096),                                                   # the last explicit one
                     _rec(kind=W.OP_QUIET, sub=caps["device_ctx_count"] - 1, issuer=1)])
    sg.run_script(dev, len(ops), None)
    ref = orc.Heap(npes, H, init)
    ref.run_script(ops)
    assert sg.get_status()[0] == 0 and first_diff(download(h), ref.mem) is None


def test_space_symmetry(sg, heapf):
    """Collective allocation gives the same offset on every PE; each PE's copy is
    addressable and holds its own data (Sec. 6.1)."""
    npes, H = 8, 1 << 20
    h = heapf(npes, H)
    objs = [h.malloc(n) for n in (1, 100, 4096, 65536, 200000)]
    offs = [o.offset for o in objs]
    assert all(o % 256 == 0 for o in offs) and len(set(offs)) == len(offs)
    for o in objs:
        for p in range(npes):
            assert h.ptr(o, p) == h.base + p * H + o.offset
    o = objs[3]
    parts = h.partitions()
    for p in range(npes):                       # a distinct pattern in every PE's copy
        parts[p, o.offset:o.offset + 65536] = p + 1
    # PE 0 gathers every PE's copy with device-initiated gets
    ops = [_rec(kind=W.OP_GET, pe=p, issuer=0, dst=objs[4].offset + 8 * KiB * p, src=o.offset, n=8 * KiB)
           for p in range(npes)]
    _, dev = _dev(ops)
    sg.run_script(dev, len(ops), None)
    torch.cuda.synchronize()
    got = parts[0, objs[4].offset:objs[4].offset + 8 * KiB * npes].cpu().numpy().reshape(npes, 8 * KiB)
    assert all((got[p] == p + 1).all() for p in range(npes))


def test_gpu_space_at_init(sg, heapf):
    """The GPU symmetric heap exists right after initialisation: reported by the
    capability query, allocatable without creating a space (Sec. 6.1)."""
    npes, H = 4, 1 << 20
    h = heapf(npes, H)
    caps = sg.query_capabilities(sg.TEAM_WORLD)
    assert caps["default_heap"] == 1 and caps["heap_bytes_per_pe"] == H and caps["heap_free_bytes"] == H
    a = h.malloc(H // 2)
    assert a.offset == 0
    assert sg.query_capabilities(sg.TEAM_WORLD)["heap_free_bytes"] == H - H // 2


def test_quiet_completes_device_operations(sg, heapf):
    """Device side: quiet completes the PE's non-blocking puts (the bulk engine's
    asynchronous copies included) before the signal that follows it, so the target
    sees all of the data once it sees the signal (Sec. 6.4)."""
    npes, H = 2, 16 << 20
    h = heapf(npes, H)
    parts = h.partitions()
    parts.zero_()
    m = 4 << 20
    sig = 3 * m
    for rnd in range(1, 6):
        parts[0, :m] = rnd                      # new payload every round
        parts[1, sig:sig + 8] = 0
        ops = [_rec(kind=W.OP_PUT_NBI, pe=1, issuer=0, dst=m, src=0, n=m),
               _rec(kind=W.OP_QUIET, issuer=0),
               _rec(kind=W.OP_PUT_SIGNAL, sub=W.SIG_SET, pe=1, issuer=0, dst=2 * m, src=0, n=16,
                    operand=rnd, aux=sig),
               _rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_EQ, issuer=1, dst=sig, operand=rnd),
               _rec(kind=W.OP_PUT, pe=1, issuer=1, dst=0, src=m, n=m)]   # PE 1 copies what arrived
        _, dev = _dev(ops)
        sg.run_script(dev, len(ops), None)
        torch.cuda.synchronize()
        assert sg.get_status()[0] == 0
        assert bool((parts[1, :m] == rnd).all())


def test_fence_orders_puts(sg, heapf):
    """fence orders a PE's later puts after its earlier ones at the target: once the
    target sees the second (a flag word), it sees the first (Sec. 6.4)."""
    npes, H = 2, 1 << 20
    h = heapf(npes, H)
    parts = h.partitions()
    for rnd in range(1, 9):
        parts[0, :64 * KiB] = rnd
        parts[0, 128 * KiB:128 * KiB + 8].view(torch.int64)[0] = rnd
        parts[1, 256 * KiB:256 * KiB + 8] = 0
        ops = [_rec(kind=W.OP_PUT, pe=1, issuer=0, dst=64 * KiB, src=0, n=64 * KiB),
               _rec(kind=W.OP_FENCE, issuer=0),
               _rec(kind=W.OP_PUT, pe=1, issuer=0, dst=256 * KiB, src=128 * KiB, n=8),
               _rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_EQ, issuer=1, dst=256 * KiB, operand=rnd),
               _rec(kind=W.OP_PUT, pe=1, issuer=1, dst=512 * KiB, src=64 * KiB, n=64 * KiB)]
        _, dev = _dev(ops)
        sg.run_script(dev, len(ops), None)
        torch.cuda.synchronize()
        assert sg.get_status()[0] == 0
        assert bool((parts[1, 512 * KiB:576 * KiB] == rnd).all())


def test_stream_ordering_host_and_device(sg, heapf, orc):
    """Within one stream, host-issued (stream-triggered) operations, device-initiated
    scripts and host collectives take effect in stream order with no synchronisation
    in between (Sec. 6.4 stream-triggered semantics)."""
    npes, H = 8, 1 << 20
    h = heapf(npes, H)
    init = random_heap(npes, H, 5)
    upload(h, init)
    torch.cuda.synchronize()
    ref = orc.Heap(npes, H, init)
    s = torch.cuda.Stream()
    b = h.base
    with torch.cuda.stream(s):
        sg.putmem(b + 4096, b + 0, 3000, 5, 2, s)                           # host put: 2 -> 5
        ref.put(4096, 0, 3000, 5, 2)
        ops, dev = _dev([_rec(kind=W.OP_GET, pe=5, issuer=7, dst=20000, src=4096, n=3000),  # device: 7 reads it
                         _rec(kind=W.OP_REDUCE, dtype=W.DT_INT64, sub=W.RED_SUM, team=0, dst=40000, src=24576, n=500)])
        sg.run_script(dev, len(ops), None, s)
        ref.run_script(ops)
        sg.reduce(sg.TEAM_WORLD, b + 60000, b + 40000, 500, sg.INT64, sg.MAX, s)   # host reduce of the device result
        ref.reduce((0, 1, npes), 60000, 40000, 500, W.DT_INT64, W.RED_MAX)
        sg.getmem(b + 80000, b + 20000, 3000, 7, 1, s)                      # host get of the device get's result
        ref.get(80000, 20000, 3000, 7, 1)
    sg.quiet(s)                                                              # host quiet = stream completion
    assert first_diff(download(h), ref.mem) is None


def test_stream_ordering_across_streams_by_event(sg, heapf, orc):
    """Two streams are ordered only by an explicit dependency: with an event, the
    second stream's get sees the first stream's put."""
    npes, H = 4, 1 << 20
    h = heapf(npes, H)
    init = random_heap(npes, H, 6)
    upload(h, init)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    b = h.base
    sg.putmem(b + 65536, b + 0, 256 * KiB, 1, 0, s1)
    ev = torch.cuda.Event()
    ev.record(s1)
    s2.wait_event(ev)
    sg.getmem(b + 400000, b + 65536, 256 * KiB, 1, 3, s2)
    sg.quiet(s2)
    ref = orc.Heap(npes, H, init)
    ref.put(65536, 0, 256 * KiB, 1, 0)
    ref.get(400000, 65536, 256 * KiB, 1, 3)
    torch.cuda.synchronize()
    assert first_diff(download(h), ref.mem) is None


def test_stream_ordering_in_a_cuda_graph(sg, heapf, orc):
    """Stream-triggered operations captured into a CUDA graph replay in stream order."""
    npes, H = 4, 1 << 18
    h = heapf(npes, H)
    init = random_heap(npes, H, 7)
    upload(h, init)
    b = h.base
    s = torch.cuda.Stream()
    def ops():
        sg.putmem(b + 8192, b + 0, 4096, 2, 0, s)
        sg.reduce(sg.TEAM_WORLD, b + 32768, b + 8192, 512, sg.INT64, sg.SUM, s)
        sg.broadcastmem(sg.TEAM_WORLD, b + 65536, b + 32768, 4096, 2, s)
    torch.cuda.synchronize()
    ops()                                    # first use outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sg.putmem(b + 8192, b + 0, 4096, 2, 0, s)
        sg.reduce(sg.TEAM_WORLD, b + 32768, b + 8192, 512, sg.INT64, sg.SUM, s)
        sg.broadcastmem(sg.TEAM_WORLD, b + 65536, b + 32768, 4096, 2, s)
    torch.cuda.synchronize()
    upload(h, init)                          # capture ran nothing; replay twice
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    ref = orc.Heap(npes, H, init)
    for _ in range(2):
        ref.put(8192, 0, 4096, 2, 0)
        ref.reduce((0, 1, npes), 32768, 8192, 512, W.DT_INT64, W.RED_SUM)
        ref.broadcast((0, 1, npes), 65536, 32768, 4096, 2)
    assert first_diff(download(h), ref.mem) is None


def test_wait_before_its_signal_in_one_stream_does_not_deadlock(sg, heapf):
    """A documented prohibited pattern: a host wait_until enqueued before the
    put_signal that would satisfy it on the same stream.  The wait is bounded, so the
    stream does not deadlock: the wait records a timeout and the signal then lands."""
    npes, H = 2, 1 << 16
    h = heapf(npes, H, timeout_ns=3_000_000)
    h.partitions().zero_()
    b = h.base
    s = torch.cuda.Stream()
    sg.clear_status(s)
    sg.signal_wait_until(b + 4096, 1, W.CMP_EQ, 1, s)
    sg.putmem_signal(b + 8192, b + 0, 64, b + 4096, 1, W.SIG_SET, 1, 0, s)
    sg.quiet(s)
    code, _ = sg.get_status()
    assert code == sg.ERR_TIMEOUT
    assert int(h.partitions()[1, 4096:4104].view(torch.int64)[0]) == 1
    sg.clear_status()


def test_mixed_host_device_collectives_are_documented(sg, heapf, orc):
    """Host and device collectives on one team are undefined without explicit ordering
    (Sec. 6.3); the capability does not claim them.  With stream order as the explicit
    ordering, a host reduce followed by a device reduce on the same team is defined."""
    npes, H = 4, 1 << 16
    h = heapf(npes, H)
    assert "MIXED_HOST_DEVICE_COLL" not in sg.query_capabilities(sg.TEAM_WORLD)["flag_names"]
    init = random_heap(npes, H, 8)
    upload(h, init)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    sg.reduce(sg.TEAM_WORLD, h.base + 8192, h.base, 256, sg.INT32, sg.SUM, s)
    ops, dev = _dev([_rec(kind=W.OP_REDUCE, dtype=W.DT_INT32, sub=W.RED_MAX, team=0, dst=16384, src=8192, n=256)])
    sg.run_script(dev, 1, None, s)
    sg.quiet(s)
    ref = orc.Heap(npes, H, init)
    ref.reduce((0, 1, npes), 8192, 0, 256, W.DT_INT32, W.RED_SUM)
    ref.run_script(ops)
    assert first_diff(download(h), ref.mem) is None


def test_pointer_accessibility(sg, heapf):
    """shmemg_ptr returns a device-domain pointer only (Sec. 6.3 pointer queries): the
    capability reports PTR_DEVICE and not PTR_HOST, and the pointer is the symmetric
    address of that PE's copy inside the device allocation."""
    npes, H = 4, 1 << 16
    h = heapf(npes, H)
    caps = sg.query_capabilities(sg.TEAM_WORLD)
    assert "PTR_DEVICE" in caps["flag_names"] and "PTR_HOST" not in caps["flag_names"]
    a = h.malloc(1024)
    for p in range(npes):
        ptr = h.ptr(a, p)
        assert ptr == h.base + p * H + a.offset
        assert h.base <= ptr < h.base + npes * H
    with pytest.raises(sg.ShmemgError) as e:
        h.ptr(h.base + H + 64, 0)               # inside PE 1's copy: not a canonical address
    assert e.value.code == sg.ERR_NOT_SYMMETRIC


def test_progress_needs_no_host(sg, heapf, orc):
    """GPU-driven progress (capability PROGRESS_GPU, not HOST_PROGRESS_REQUIRED): a
    device script whose PEs hand a token around with put_signal / wait_until completes
    in one launch while the host only waits."""
    npes, H = 8, 1 << 16
    h = heapf(npes, H)
    caps = sg.query_capabilities(sg.TEAM_WORLD)
    assert "PROGRESS_GPU" in caps["flag_names"] and "HOST_PROGRESS_REQUIRED" not in caps["flag_names"]
    init = random_heap(npes, H, 9)
    init.reshape(npes, H)[:, 60000:60008] = 0
    upload(h, init)
    ops = []
    for p in range(npes - 1):                  # PE p passes the token to PE p+1
        if p > 0:
            ops.append(_rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_GE, issuer=p, dst=60000, operand=1))
        ops.append(_rec(kind=W.OP_PUT_SIGNAL, sub=W.SIG_ADD, pe=p + 1, issuer=p, dst=1024 * (p + 1), src=1024 * p,
                        n=1024, operand=1, aux=60000))
    ops.append(_rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_GE, issuer=npes - 1, dst=60000, operand=1))
    ops, dev = _dev(ops)
    sg.run_script(dev, len(ops), None)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(npes, H, init)
    ref.run_script(ops)
    assert first_diff(download(h), ref.mem) is None
