"""Edge cases of the GPU path against the oracle: empty operations (host-issued and in
device scripts, every kind and context), transfers and reductions of a whole partition,
the last word of a partition, signal-only put_signal and already-satisfied waits."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu


def _rec(**kw):
    r = np.zeros((), dtype=W.OP_DTYPE)
    r["issuer"] = -1
    for k, v in kw.items():
        r[k] = v
    return r


def test_empty_host_operations_change_nothing(sg, heapf):
    npes, H = 4, 1 << 16
    h = heapf(npes, H)
    init = random_heap(npes, H, 61)
    upload(h, init)
    b = h.base
    sg.putmem(b + 64, b + 4096, 0, 1, 0)
    sg.getmem(b + 64, b + 4096, 0, 1, 0)
    sg.putmem(b + 64, b + 4096, 0, 1, 0, nbi=True)
    for dt in (sg.INT32, sg.INT64, sg.FLOAT):
        sg.reduce(sg.TEAM_WORLD, b + 8192, b + 0, 0, dt, sg.SUM)
    sg.broadcastmem(sg.TEAM_WORLD, b + 8192, b + 0, 0, 2)
    sg.fcollectmem(sg.TEAM_WORLD, b + 8192, b + 0, 0)
    sg.alltoallmem(sg.TEAM_WORLD, b + 8192, b + 0, 0)
    sg.quantize(sg.TEAM_WORLD, b + 16384, b + 20480, b + 0, sg.FMT_BF16, 0)
    sg.qsum_reduce(sg.TEAM_WORLD, b + 24576, b + 16384, b + 20480, sg.FMT_BF16, 0)
    sg.quiet()
    assert sg.get_status()[0] == 0
    assert first_diff(download(h), init) is None


@pytest.mark.parametrize("mode,cd", [(0, 1), (0, 2), (1, 2)])
def test_empty_device_operations_change_nothing(sg, heapf, orc, mode, cd):
    npes, H = 4, 1 << 16
    h = heapf(npes, H, pe_mode=mode, cluster_dim=cd)
    init = random_heap(npes, H, 62)
    upload(h, init)
    ops = []
    for ctx in range(4):
        ops += [_rec(kind=W.OP_PUT_NBI, sub=ctx, pe=1, issuer=0, dst=64, src=4096, n=0),
                _rec(kind=W.OP_GET_NBI, sub=ctx, pe=2, issuer=3, dst=64, src=4096, n=0)]
    ops += [_rec(kind=W.OP_PUT, pe=1, issuer=0, dst=64, src=4096, n=0),
            _rec(kind=W.OP_GET, pe=1, issuer=0, dst=64, src=4096, n=0),
            _rec(kind=W.OP_PUT | W.OP_WARP, pe=1, issuer=0, dst=64, src=4096, n=0),
            _rec(kind=W.OP_REDUCE, dtype=W.DT_INT64, sub=W.RED_SUM, team=0, dst=8192, src=0, n=0),
            _rec(kind=W.OP_REDUCE, dtype=W.DT_FLOAT, sub=W.RED_SUM, team=1, dst=8192, src=0, n=0),
            _rec(kind=W.OP_BCAST, team=0, pe=1, dst=8192, src=0, n=0),
            _rec(kind=W.OP_FCOLLECT, team=1, dst=8192, src=0, n=0),
            _rec(kind=W.OP_ALLTOALL, team=0, dst=8192, src=0, n=0),
            _rec(kind=W.OP_QUIET, sub=0xFF, issuer=-1)]
    ops = np.array(ops, dtype=W.OP_DTYPE)
    sg.clear_status()
    sg.run_script(torch.from_numpy(ops.view(np.uint8).copy()).cuda(), len(ops), None)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    assert first_diff(download(h), init) is None


def test_whole_partition_transfers_and_reduction(sg, heapf, orc):
    """A put and a get of exactly H bytes (the largest range a partition has), and an
    in-place int64 sum over the whole partition, host-issued and device-initiated."""
    npes, H = 4, 1 << 20
    h = heapf(npes, H)
    init = random_heap(npes, H, 63)
    upload(h, init)
    ref = orc.Heap(npes, H, init)
    b = h.base
    sg.putmem(b, b, H, 1, 0)           # PE 0's whole partition -> PE 1
    ref.put(0, 0, H, 1, 0)
    sg.getmem(b, b, H, 1, 2)           # PE 2 reads all of PE 1
    ref.get(0, 0, H, 1, 2)
    sg.reduce(sg.TEAM_WORLD, b, b, H // 8, sg.INT64, sg.SUM)   # in place, every word
    ref.reduce((0, 1, npes), 0, 0, H // 8, W.DT_INT64, W.RED_SUM)
    sg.quiet()
    assert first_diff(download(h), ref.mem) is None
    ops = np.array([_rec(kind=W.OP_PUT_NBI, sub=1, pe=3, issuer=2, dst=0, src=0, n=H),
                    _rec(kind=W.OP_QUIET, sub=1, issuer=2), _rec(kind=W.OP_BARRIER_ALL),
                    _rec(kind=W.OP_REDUCE, dtype=W.DT_INT32, sub=W.RED_MAX, team=0, dst=0, src=0, n=H // 4)],
                   dtype=W.OP_DTYPE)
    sg.run_script(torch.from_numpy(ops.view(np.uint8).copy()).cuda(), len(ops), None)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref.run_script(ops)
    assert first_diff(download(h), ref.mem) is None


def test_last_word_amos_signal_only_and_satisfied_waits(sg, heapf, orc):
    npes, H = 2, 1 << 16
    h = heapf(npes, H)
    init = random_heap(npes, H, 64)
    init.reshape(npes, H)[:, H - 16:H - 8] = 0           # a signal word
    upload(h, init)
    ops = np.array([
        _rec(kind=W.OP_FADD, dtype=W.DT_INT64, pe=1, issuer=0, dst=H - 8, operand=5),       # last int64 word
        _rec(kind=W.OP_FXOR, dtype=W.DT_INT32, pe=0, issuer=1, dst=H - 4, operand=0x55),    # last int32 word
        _rec(kind=W.OP_PUT_SIGNAL, sub=W.SIG_SET, pe=1, issuer=0, dst=0, src=0, n=0, operand=9, aux=H - 16),  # signal only
        _rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_EQ, issuer=1, dst=H - 16, operand=9),
        _rec(kind=W.OP_WAIT_UNTIL, sub=W.CMP_GE, issuer=1, dst=H - 16, operand=0),          # already true
        _rec(kind=W.OP_BARRIER_ALL)], dtype=W.OP_DTYPE)
    fetched = torch.zeros(len(ops), dtype=torch.int64, device="cuda")
    sg.run_script(torch.from_numpy(ops.view(np.uint8).copy()).cuda(), len(ops), fetched)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    ref = orc.Heap(npes, H, init)
    want = ref.run_script(ops)
    assert first_diff(download(h), ref.mem) is None
    got = fetched.cpu().numpy()
    assert got[0] == want[0] and (got[1] & 0xFFFFFFFF) == (want[1] & 0xFFFFFFFF)


def test_team_ranges_past_int32_are_rejected(sg, heapf):
    """A team whose start + size passes INT32_MAX is refused before anything launches
    (the range check is done in 64 bits), by the batched engine and its allocation-free
    form alike; the heap stays as it was."""
    h = heapf(4, 1 << 16)
    parts = h.partitions()
    parts.random_(0, 255)
    before = parts.clone()
    big = (1 << 31) - 1
    for start, size in ((big, 1), (1, big), (big, big)):
        d = [sg.CollDesc(start, size, sg.INT64, -1, 8, h.base + 4096, h.base, None)]
        with pytest.raises(sg.ShmemgError) as e:
            sg.Batch(d, sg.Tune(16384, 0, 0, 0))
        assert e.value.code == sg.ERR_INVALID_ARG
        with pytest.raises(sg.ShmemgError) as e:
            sg.batch_reduce_noalloc(d, 128)
        assert e.value.code == sg.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0 and torch.equal(parts, before)
