"""GPU parity of the plain path: every host-issued (stream-triggered) operation and the
device-initiated script interpreter against the CPU oracle, bit-exact heaps."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu


def test_init_caps_malloc_ptr(sg, heapf, orc):
    h = heapf(6, 1 << 16, pe_mode=sg.PE_MODE_CTA, cluster_dim=2)
    caps = sg.query_capabilities(sg.TEAM_WORLD)
    for f in ("GPU_AWARE_HOST", "DEVICE_RMA", "DEVICE_AMO", "DEVICE_COLL", "DEVICE_CTX_DEFAULT", "DEVICE_TEAMS",
              "PTR_DEVICE", "STREAM_ORDERED", "PROGRESS_GPU"):
        assert f in caps["flag_names"]
    assert "PTR_HOST" not in caps["flag_names"] and "EXPLICIT_DEVICE_CTX" in caps["flag_names"]
    assert caps["device_ctx_count"] == 4
    assert caps["team_n_pes"] == 6 and caps["shared_team_size"] == 2 and caps["default_heap"] == 1
    assert sg.query_capabilities(sg.TEAM_SHARED)["team_n_pes"] == 2
    a = h.malloc(100)
    b = h.malloc(1000)
    assert a.offset % 256 == 0 and b.offset % 256 == 0 and b.offset >= a.offset + 256
    # symmetric: PE p's copy is at base + p*H + offset, for every p
    for p in range(6):
        assert h.ptr(b, p) == h.base + p * h.H + b.offset
    h.free(a)
    c = h.malloc(64)
    assert c.offset == a.offset          # first fit reuses the freed range
    with pytest.raises(sg.ShmemgError) as e:
        h.malloc(1 << 20)
    assert e.value.code == sg.ERR_OUT_OF_HEAP
    with pytest.raises(sg.ShmemgError) as e:
        sg.putmem(h.base + h.H - 8, a.ptr, 16, 1, 0)   # range leaves the partition
    assert e.value.code == sg.ERR_NOT_SYMMETRIC
    with pytest.raises(sg.ShmemgError):
        sg.putmem(a.ptr, b.ptr, 8, 6, 0)              # PE out of range
    t = sg.team_split_strided(sg.TEAM_WORLD, 1, 2, 3)  # PEs 1, 3, 5
    assert sg.team_n_pes(t) == 3 and sg.team_translate_pe(t, 2, sg.TEAM_WORLD) == 5
    assert sg.team_translate_pe(sg.TEAM_WORLD, 3, t) == 1 and sg.team_translate_pe(sg.TEAM_WORLD, 2, t) == -1
    sg.team_destroy(t)


@pytest.mark.parametrize("n,dst,src", [(1, 3, 100), (7, 8, 1), (8, 16, 24), (4096, 4096, 0), (4095, 512, 8),
                                       (65536 + 8, 1024, 200000), (1 << 20, 0, 1 << 21)])
def test_put_get_sizes_alignments(sg, heapf, orc, n, dst, src):
    npes, H = 3, 4 << 20
    h = heapf(npes, H)
    init = random_heap(npes, H, 7 + n)
    upload(h, init)
    ref = orc.Heap(npes, H, init)
    sg.putmem(h.base + dst, h.base + src, n, 2, 0)
    ref.put(dst, src, n, 2, 0)
    sg.getmem(h.base + src, h.base + dst, n, 2, 1, nbi=True)     # back into PE 1
    ref.get(src, dst, n, 2, 1)
    d2 = (3 << 20) + dst % 16
    sg.putmem(h.base + d2, h.base + src, n // 2, 0, 0, nbi=True)  # PE0 -> PE0, disjoint ranges
    ref.put(d2, src, n // 2, 0, 0)
    sg.quiet()
    got = download(h)
    assert first_diff(got, ref.mem) is None


def test_host_amos_and_signals(sg, heapf, orc):
    npes, H = 4, 1 << 16
    h = heapf(npes, H)
    init = random_heap(npes, H, 99)
    upload(h, init)
    ref = orc.Heap(npes, H, init)
    fetched = torch.zeros(64, dtype=torch.int64, device="cuda")
    rng = W.SplitMix64(5)
    want = []
    for i in range(40):
        kind = ["fetch_add", "compare_swap", "fetch_xor"][i % 3]
        pe, off = rng.below(npes), 8 * rng.below(4)      # few words: heavy reuse, script order
        v = rng.next() - (1 << 63)
        cond = int(ref.view(pe, off, 1, np.int64)[0]) if i % 2 else 5
        sg.atomic(kind, sg.INT64, h.base + off, v, pe, fetched=fetched.data_ptr() + 8 * i, cond=cond)
        k = {"fetch_add": W.OP_FADD, "compare_swap": W.OP_CSWAP, "fetch_xor": W.OP_FXOR}[kind]
        want.append(ref.amo64(k, pe, off, v, cond))
    f32 = torch.zeros(8, dtype=torch.int32, device="cuda")
    sg.atomic("fetch_add", sg.INT32, h.base + 4096 + 4, 2**31 - 1, 1, fetched=f32.data_ptr())
    w32 = ref.amo32(W.OP_FADD, 1, 4096 + 4, 2**31 - 1)
    # put with signal (ADD) then a stream-ordered wait on the target's signal
    sig = 8192
    sg.putmem_signal(h.base + 10000, h.base + 20000, 3000, h.base + sig, 5, sg.SIGNAL_ADD, 3, 2)
    ref.put_signal(10000, 20000, 3000, sig, W.SIG_ADD, 5, 3, 2)
    cur = int(ref.view(3, sig, 1, np.uint64)[0])
    sg.signal_wait_until(h.base + sig, 3, sg.CMP_EQ, cur)
    sg.putmem_signal(h.base + 30000, h.base + 20000, 1 << 15, h.base + sig, 77, sg.SIGNAL_SET, 0, 1)
    ref.put_signal(30000, 20000, 1 << 15, sig, W.SIG_SET, 77, 0, 1)
    sg.quiet()
    assert fetched[:40].cpu().tolist() == want
    assert int(f32[0]) == w32
    assert first_diff(download(h), ref.mem) is None
    assert sg.get_status()[0] == 0


def test_wait_timeout_sets_status(sg, heapf):
    h = heapf(2, 4096, timeout_ns=2_000_000)   # 2 ms
    sig = h.calloc(8)
    sg.quiet()
    sg.clear_status()
    sg.signal_wait_until(sig, 1, sg.CMP_EQ, 1)  # nothing ever sets it
    sg.quiet()
    code, _ = sg.get_status()
    assert code == sg.ERR_TIMEOUT
    sg.clear_status()
    assert sg.get_status()[0] == 0


TEAMS = [("world", None), ("split", (1, 2, 3)), ("single", (2, 1, 1))]


@pytest.mark.parametrize("npes", [1, 5, 8])
@pytest.mark.parametrize("n", [1, 7, 4095, 4096 + 3])
def test_reduce_all_types(sg, heapf, orc, npes, n):
    H = 1 << 17
    h = heapf(npes, H)
    for dtype, npdt, es in [(sg.INT32, np.int32, 4), (sg.INT64, np.int64, 8), (sg.FLOAT, np.float32, 4)]:
        init = random_heap(npes, H, n * 31 + dtype)
        hv = init.view(np.uint8).reshape(npes, H)
        if dtype == sg.FLOAT:   # finite floats: N(0,1) payloads at both src offsets
            for p in range(npes):
                hv[p, 0:8 * n] = W.normals_np(p + 17 * n, 2 * n).astype(np.float32).view(np.uint8)
                hv[p, 40000:40000 + 4 * n] = W.normals_np(p + 3, n).astype(np.float32).view(np.uint8)
        upload(h, init)
        ref = orc.Heap(npes, H, init)
        for op in (sg.SUM, sg.MAX, sg.MIN):
            for name, tspec in TEAMS:
                if tspec and tspec[0] + (tspec[2] - 1) * tspec[1] >= npes:
                    continue
                team = sg.TEAM_WORLD if tspec is None else sg.team_split_strided(sg.TEAM_WORLD, *tspec)
                tt = (0, 1, npes) if tspec is None else tspec
                dst = 65536 + 16 * op + (8 if n % 2 else 0)   # vector and scalar paths
                sg.reduce(team, h.base + dst, h.base + 0, n, dtype, op)
                ref.reduce(tt, dst, 0, n, dtype, op)
                if tspec is not None:
                    sg.team_destroy(team)
            # in place
            sg.reduce(sg.TEAM_WORLD, h.base + 40000, h.base + 40000, n, dtype, op)
            ref.reduce((0, 1, npes), 40000, 40000, n, dtype, op)
        got = download(h)
        assert first_diff(got, ref.mem) is None, (dtype, first_diff(got, ref.mem))


@pytest.mark.parametrize("npes", [1, 3, 64])
def test_broadcast_fcollect_alltoall(sg, heapf, orc, npes):
    H = 1 << 18
    h = heapf(npes, H)
    init = random_heap(npes, H, npes)
    upload(h, init)
    ref = orc.Heap(npes, H, init)
    for n in (1, 24, 1000, 4096):
        if n * npes * 2 > H // 2:
            continue
        root = npes - 1
        sg.broadcastmem(sg.TEAM_WORLD, h.base + 100000, h.base + 8, n, root)
        ref.broadcast((0, 1, npes), 100000, 8, n, root)
        sg.fcollectmem(sg.TEAM_WORLD, h.base + 0, h.base + 200000, n)
        ref.fcollect((0, 1, npes), 0, 200000, n)
        m = max(1, n // 4)
        sg.alltoallmem(sg.TEAM_WORLD, h.base + 150000 - m * npes, h.base + 16, m)
        ref.alltoall((0, 1, npes), 150000 - m * npes, 16, m)
    if npes >= 3:
        t = sg.team_split_strided(sg.TEAM_WORLD, 0, 2, (npes + 1) // 2)
        sg.broadcastmem(t, h.base + 4096, h.base + 120000, 777, 1)
        ref.broadcast((0, 2, (npes + 1) // 2), 4096, 120000, 777, 1)
        sg.alltoallmem(t, h.base + 64, h.base + 210000, 40, )
        ref.alltoall((0, 2, (npes + 1) // 2), 64, 210000, 40)
        sg.team_destroy(t)
    sg.quiet()
    assert first_diff(download(h), ref.mem) is None


def test_shared_team_groups(sg, heapf, orc):
    npes, H = 8, 1 << 14
    h = heapf(npes, H, pe_mode=sg.PE_MODE_CTA, cluster_dim=4)
    init = random_heap(npes, H, 3)
    upload(h, init)
    ref = orc.Heap(npes, H, init)
    sg.reduce(sg.TEAM_SHARED, h.base + 4096, h.base + 0, 100, sg.INT64, sg.SUM)
    sg.broadcastmem(sg.TEAM_SHARED, h.base + 8192, h.base + 1000, 300, 3)
    for g in range(2):   # one collective per cluster group of 4 PEs
        ref.reduce((4 * g, 1, 4), 4096, 0, 100, W.DT_INT64, W.RED_SUM)
        ref.broadcast((4 * g, 1, 4), 8192, 1000, 300, 3)
    assert first_diff(download(h), ref.mem) is None


def _script_heap(sg, heapf, s, **kw):
    h = heapf(s.npes, s.heap_bytes, **kw)
    upload(h, s.heap)
    return h


def test_plain_script_host_path_strict(sg, heapf, orc):
    """Launch-per-op path on a script WITH conflicts: script order, bit-exact."""
    s = W.gen_plain_script(seed=4242, n_ops=3000, race_free=False)
    h = _script_heap(sg, heapf, s)
    fetched = torch.zeros(len(s.ops), dtype=torch.int64, device="cuda")
    sg.run_script_host(s.ops, fetched)
    sg.quiet()
    ref = orc.Heap(s.npes, s.heap_bytes, s.heap)
    want = ref.run_script(s.ops)
    amo = np.isin(s.ops["kind"], W.AMO_KINDS)
    assert np.array_equal(fetched.cpu().numpy()[amo], want[amo])
    assert first_diff(download(h), ref.mem) is None


@pytest.mark.parametrize("mode,cd", [(0, 1), (0, 2), (1, 2)])
def test_plain_script_device_initiated(sg, heapf, orc, mode, cd):
    """The 4-PE x 1 MiB, 10,000-op script through the device-initiated interpreter:
    final heap bit-exact, fetched values a valid serialisation per sync interval."""
    s = W.gen_plain_script()
    h = _script_heap(sg, heapf, s, pe_mode=mode, cluster_dim=cd)
    ops = torch.from_numpy(s.ops.view(np.uint8).copy()).cuda()
    fetched = torch.zeros(len(s.ops), dtype=torch.int64, device="cuda")
    sg.run_script(ops, len(s.ops), fetched)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(s.npes, s.heap_bytes, s.heap)
    want = ref.run_script(s.ops)
    assert first_diff(download(h), ref.mem) is None
    got = fetched.cpu().numpy()
    ids = W.sync_interval_ids(s.ops)
    idx = np.nonzero(np.isin(s.ops["kind"], W.AMO_KINDS))[0]
    group = ids[idx] * (s.npes * s.heap_bytes) + s.ops["pe"][idx].astype(np.int64) * s.heap_bytes + \
        s.ops["dst"][idx].astype(np.int64)
    firsts = {}
    w0 = np.array([firsts.setdefault(g, want[i]) for g, i in zip(group, idx)], np.int64)
    assert orc.check_serialisation(group, s.ops["kind"][idx], s.ops["operand"][idx], s.ops["cond"][idx],
                                   got[idx], w0) == 0
    # words hit once per interval must match the sequential fetched value exactly
    uniq, cnt = np.unique(group, return_counts=True)
    single = np.isin(group, uniq[cnt == 1])
    assert np.array_equal(got[idx][single], want[idx][single])


def test_device_script_collectives_signals(sg, heapf, orc):
    """Device-initiated fcollect / alltoall / float reduce / put_signal + wait_until."""
    npes, H = 6, 1 << 16
    h = heapf(npes, H)
    init = random_heap(npes, H, 11)
    init.reshape(npes, H)[:, 0:4096] = W.normals_np(1, npes * 1024).astype(np.float32).view(np.uint8).reshape(npes, 4096)
    init.reshape(npes, H)[:, 60000:60064] = 0       # signal words
    upload(h, init)
    t = sg.team_split_strided(sg.TEAM_WORLD, 1, 1, 5)
    ops = np.zeros(9, W.OP_DTYPE)
    ops[0] = (W.OP_REDUCE, W.DT_FLOAT, W.RED_SUM, 0, 0, -1, 8192, 0, 1000, 0, 0, 0)
    ops[1] = (W.OP_FCOLLECT, 0, 0, t, 0, -1, 16384, 4096, 600, 0, 0, 0)
    ops[2] = (W.OP_ALLTOALL, 0, 0, 0, 0, -1, 32768, 12288, 320, 0, 0, 0)
    ops[3] = (W.OP_PUT_SIGNAL, 0, W.SIG_ADD, 0, 4, 1, 50000, 20000, 1000, 3, 0, 60000)
    ops[4] = (W.OP_WAIT_UNTIL, 0, W.CMP_GE, 0, 0, 4, 60000, 0, 0, 3, 0, 0)
    ops[5] = (W.OP_GET, 0, 0, 0, 4, 5, 52000, 50000, 1000, 0, 0, 0)   # after the wait? no: issuer 5
    ops[6] = (W.OP_BARRIER_ALL, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0)
    ops[7] = (W.OP_BCAST, 0, 0, t, 2, -1, 40000, 50000, 1000, 0, 0, 0)
    ops[8] = (W.OP_REDUCE, W.DT_INT32, W.RED_MAX, t, 0, -1, 24000, 100, 333, 0, 0, 0)
    # op 5 (PE 5 reads PE 4's 50000) races with op 3 unless ordered: move it after the barrier
    ops = ops[[0, 1, 2, 3, 4, 6, 5, 7, 8]]
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    fetched = torch.zeros(len(ops), dtype=torch.int64, device="cuda")
    sg.run_script(dev, len(ops), fetched)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(npes, H, init)
    ref.run_script(ops, teams=[(0, 1, npes), (0, 1, 1), (1, 1, 5)][:t] + [(1, 1, 5)])
    assert first_diff(download(h), ref.mem) is None
    sg.team_destroy(t)


def test_device_barrier_timeout_is_bounded(sg, heapf):
    """A wait that nothing satisfies ends with a timeout status; the context survives."""
    npes, H = 2, 4096
    h = heapf(npes, H, timeout_ns=3_000_000)
    ops = np.zeros(1, W.OP_DTYPE)
    ops[0] = (W.OP_WAIT_UNTIL, 0, W.CMP_EQ, 0, 0, 1, 0, 0, 0, 12345, 0, 0)
    h.partitions().zero_()
    sg.clear_status()
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    sg.run_script(dev, 1, None)
    torch.cuda.synchronize()
    code, detail = sg.get_status()
    assert code == sg.ERR_TIMEOUT and detail == 0
    sg.clear_status()
    x = torch.ones(4, device="cuda")
    assert float(x.sum()) == 4.0


def test_device_script_rejects_invalid_op(sg, heapf, orc):
    """An op outside the heap stops the device-initiated script at that op; the status
    word names it and the ops before it have run."""
    npes, H = 4, 1 << 16
    h = heapf(npes, H)
    init = random_heap(npes, H, 5)
    upload(h, init)
    ops = np.zeros(5, W.OP_DTYPE)
    ops[0] = (W.OP_PUT, 0, 0, 0, 1, 0, 4096, 0, 512, 0, 0, 0)
    ops[1] = (W.OP_BARRIER_ALL, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0)
    ops[2] = (W.OP_FADD, W.DT_INT64, 0, 0, 2, 3, 8192, 0, 0, 7, 0, 0)
    ops[3] = (W.OP_PUT, 0, 0, 0, 9, 0, 0, 0, 8, 0, 0, 0)            # PE 9 does not exist
    ops[4] = (W.OP_PUT, 0, 0, 0, 2, 1, 0, 0, 8, 0, 0, 0)
    sg.clear_status()
    dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    fetched = torch.zeros(5, dtype=torch.int64, device="cuda")
    sg.run_script(dev, 5, fetched)
    torch.cuda.synchronize()
    code, detail = sg.get_status()
    assert code == sg.ERR_INVALID_ARG and detail == 3
    sg.clear_status()
    ref = orc.Heap(npes, H, init)
    want = ref.run_script(ops[:3])
    assert first_diff(download(h), ref.mem) is None
    assert int(fetched[2]) == want[2]
