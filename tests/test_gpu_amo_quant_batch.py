"""GPU parity of the AMO stress stream, put-signal ping-pong, quantised payloads and
the batched persistent engine against the CPU oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import download, first_diff, random_heap, upload

pytestmark = pytest.mark.gpu


def _table_heap(heapf, npes, wpp, tseed):
    H = (wpp * 8 + 255) // 256 * 256 + 65536
    h = heapf(npes, H)
    init = W.cb64_np(tseed, np.arange(npes * wpp, dtype=np.uint64)).view(np.int64)
    parts = h.partitions()
    parts[:, :wpp * 8].copy_(torch.from_numpy(init.view(np.uint8).reshape(npes, wpp * 8)).cuda())
    return h, init


def _check_stream(sg, orc, h, init, ops, wpp, oseed, tseed, agg):
    npes = h.npes
    nops = len(ops)
    dops = torch.from_numpy(ops.view(np.int32)).cuda()
    fetched = torch.zeros(nops, dtype=torch.int64, device="cuda")
    sg.amo_stream(h.base, wpp, dops, nops, oseed, tseed, fetched, flags=agg)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    final = h.partitions()[:, :wpp * 8].contiguous().view(torch.int64).reshape(-1).cpu().numpy()
    f = fetched.cpu().numpy()
    w = (ops & ((1 << 27) - 1)).astype(np.int64)
    code = (ops >> 27) & 3
    kind = np.array([W.OP_FADD, W.OP_CSWAP, W.OP_FXOR])[code]
    r = W.cb64_np(oseed, np.arange(nops, dtype=np.uint64))
    operand = np.where(code == 0, (r % np.uint64(1 << 20)) + np.uint64(1), np.where(r == 0, np.uint64(1), r)).view(np.int64)
    cond = init[w]
    bad = orc.check_serialisation(w, kind, operand, cond, f, init[w], final[w])
    assert bad == 0
    # words never touched keep their value
    untouched = np.setdiff1d(np.arange(npes * wpp), w)
    assert np.array_equal(final[untouched], init[untouched])


@pytest.mark.parametrize("agg", [0, 1, 2])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_amo_stream_serialisation(sg, heapf, orc, agg, dist):
    npes, wpp = 64, 1024
    tseed, oseed = 0x1234, 0x9876
    h, init = _table_heap(heapf, npes, wpp, tseed)
    _check_stream(sg, orc, h, init, W.amo_stream_np(77, 1 << 18, 16, dist=dist), wpp, oseed, tseed, agg)


@pytest.mark.parametrize("agg", [1, 2])
def test_amo_stream_hot_words_ragged(sg, heapf, orc, agg):
    """A few hot words (Zipf over 64 words), a stream whose length divides neither the
    PE count nor the 1024-op combining tile, and op seed == table seed so that the
    compare_swap ops i that target word i swap in exactly their compare value (applied
    outside any group by the combining kernel)."""
    npes, wpp = 8, 8
    seed = 0x5EED
    h, init = _table_heap(heapf, npes, wpp, seed)
    nops = 3 * 8 * 1024 + 777
    ops = W.amo_stream_np(91, nops, 6, dist="zipf")
    solo = np.arange(0, npes * wpp, dtype=np.uint32)
    ops[solo] = solo | np.uint32(W.AMO_CODE_CSWAP << W.AMO_WORD_BITS)
    _check_stream(sg, orc, h, init, ops, wpp, seed, seed, agg)


@pytest.mark.parametrize("agg", [1, 2])
def test_amo_stream_single_kind_exact(sg, heapf, orc, agg):
    npes, wpp = 16, 4096
    tseed, oseed = 5, 6
    for only in (W.AMO_CODE_FADD, W.AMO_CODE_FXOR):
        h, init = _table_heap(heapf, npes, wpp, tseed)
        nops = 300001
        ops = W.amo_stream_np(3, nops, 16, only=only)
        dops = torch.from_numpy(ops.view(np.int32)).cuda()
        sg.amo_stream(h.base, wpp, dops, nops, oseed, tseed, None, flags=agg)
        torch.cuda.synchronize()
        table = init.copy()
        orc.amo_stream(table, ops, oseed, tseed, want_fetched=False)
        final = h.partitions()[:, :wpp * 8].contiguous().view(torch.int64).reshape(-1).cpu().numpy()
        assert np.array_equal(final, table)    # order-independent: bit-exact
        h.close()


@pytest.mark.parametrize("agg", [0, 2])
def test_amo_stream_bounds_error(sg, heapf, agg):
    npes, wpp = 4, 256
    h, _ = _table_heap(heapf, npes, wpp, 1)
    ops = np.array([5, 1023 | (1 << 27), 2000, 7 | (3 << 27)], dtype=np.uint32)
    sg.clear_status()
    sg.amo_stream(h.base, wpp, torch.from_numpy(ops.view(np.int32)).cuda(), 4, 1, 1, None, flags=agg)
    torch.cuda.synchronize()
    code, detail = sg.get_status()
    assert code == sg.ERR_INVALID_ARG and detail in (2, 3)
    sg.clear_status()


@pytest.mark.parametrize("payload", [8, 100, 4096])
def test_pingpong_final_state(sg, heapf, orc, payload):
    npairs, iters, npes = 16, 200, 32
    H = 3 * 4096 + 256
    h = heapf(npes, H)
    init = random_heap(npes, H, payload)
    init.reshape(npes, H)[:, 3 * 4096:3 * 4096 + 8] = 0
    upload(h, init)
    lat = torch.zeros(npairs * iters, dtype=torch.int64, device="cuda")
    sg.pingpong(h.base, h.base + 3 * 4096, payload, npairs, iters, lat)
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


def _fill_floats(h, off, n, seed, scale=1.0, special=False):
    x = (W.normals_np(seed, h.npes * n) * scale).astype(np.float32).reshape(h.npes, n)
    if special and n >= 256:
        x[:, 128:256] = 0.0                       # an all-zero block: scale 1
        x[0, 0:8] = [448.0, -448.0, 1.0625, 1.1875, 0.0146484375, 1e-9, -3e-3, 2.0 ** -10]
    for p in range(h.npes):
        h.view(off, p, torch.float32, n).copy_(torch.from_numpy(x[p]))
    return x


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("npes,n", [(1, 300), (3, 1000), (64, 4096 + 17), (5, 128)])
def test_quantize_and_qsum_bitexact(sg, heapf, orc, fmt, npes, n):
    H = 1 << 17
    h = heapf(npes, H)
    xo, qo, so, do = 0, 32768, 65536, 81920
    _fill_floats(h, xo, n, 7 * n + npes, scale=5.0, special=True)
    torch.cuda.synchronize()
    init = download(h)
    sg.quantize(sg.TEAM_WORLD, h.base + qo, h.base + so, h.base + xo, fmt, n)
    sg.qsum_reduce(sg.TEAM_WORLD, h.base + do, h.base + qo, h.base + so, fmt, n)
    torch.cuda.synchronize()
    got = download(h)
    ref = orc.Heap(npes, H, init)
    qs = 1 if fmt else 2
    for p in range(npes):
        q, s = orc.quantize(ref.view(p, xo, n, np.float32).copy(), fmt)
        ref.pe(p)[qo:qo + n * qs] = q.view(np.uint8)
        ref.pe(p)[so:so + 4 * len(s)] = s.view(np.uint8)
    ref.qsum_reduce((0, 1, npes), do, qo, so, fmt, n)
    g = got.reshape(npes, H)
    r = ref.mem.reshape(npes, H)
    assert np.array_equal(g[:, qo:qo + n * qs], r[:, qo:qo + n * qs]), "codes differ"
    assert np.array_equal(g[:, so:so + 4 * ((n + 127) // 128)], r[:, so:so + 4 * ((n + 127) // 128)]), "scales differ"
    assert np.array_equal(g[:, do:do + 4 * n], r[:, do:do + 4 * n]), "compensated sums differ"
    # accumulation error vs the binary64 sum of the dequantised payloads (gated)
    y = r[0, do:do + 4 * n].view(np.float32).astype(np.float64)
    y64, a64 = ref.qsum_ref64((0, 1, npes), qo, so, fmt, n)
    u = 2.0 ** -24
    assert np.all(np.abs(y - y64) <= 2 * u * np.abs(y64) + 2 * npes * npes * u * u * a64 + 1e-45)


def test_batch_engine_bitexact_and_replay(sg, heapf, orc):
    world = 32
    bt = W.gen_batch_teams(seed=99, n_teams=24, world=world, p_hi=32, n_lo=100, n_hi=20000)
    fmts = [-1, -1, 0, 1]
    H = 4 << 20
    h = heapf(world, H)
    descs, layout = [], []
    for t in range(len(bt.size)):
        n = int(bt.n[t])
        if bt.is_int[t]:
            src, dst = h.malloc(8 * n), h.malloc(8 * n)
            descs.append(sg.CollDesc(int(bt.start[t]), int(bt.size[t]), sg.INT64, -1, n, dst.ptr, src.ptr, None))
            layout.append(("i64", src, dst, None, n))
        else:
            fmt = fmts[t % 4]
            qs = 4 if fmt < 0 else (2 if fmt == 0 else 1)
            src, dst = h.malloc(qs * n), h.malloc(4 * n)
            sc = h.malloc(4 * ((n + 127) // 128)) if fmt >= 0 else None
            descs.append(sg.CollDesc(int(bt.start[t]), int(bt.size[t]), sg.FLOAT, fmt, n, dst.ptr, src.ptr,
                                     sc.ptr if sc else None))
            layout.append((fmt, src, dst, sc, n))
    # inputs: int64 values, N(0,1) floats; quantised teams get codes from the library's
    # quantizer (checked bit-exact above) applied to per-PE floats
    tmpf = h.malloc(4 * 20000)
    for (kind, src, dst, sc, n), t in zip(layout, range(len(layout))):
        if kind == "i64":
            v = W.uniform_ints_np(t, np.arange(world * n, dtype=np.uint64), -(1 << 20), 1 << 20).reshape(world, n)
            for p in range(world):
                h.view(src, p, torch.int64, n).copy_(torch.from_numpy(v[p]))
        elif kind == -1:
            _fill_floats(h, src.offset, n, 1000 + t)
        else:
            _fill_floats(h, tmpf.offset, n, 2000 + t)
            sg.quantize(sg.TEAM_WORLD, src, sc, tmpf, kind, n)
    torch.cuda.synchronize()
    init = download(h)
    b = sg.Batch(descs, sg.Tune(4096, 0, 0, 0))
    b.launch()
    torch.cuda.synchronize()
    got1 = download(h)
    ref = orc.Heap(world, H, init)
    for (kind, src, dst, sc, n), t in zip(layout, range(len(layout))):
        team = (int(bt.start[t]), 1, int(bt.size[t]))
        if kind == "i64":
            ref.reduce(team, dst.offset, src.offset, n, W.DT_INT64, W.RED_SUM)
        elif kind == -1:
            ref.reduce(team, dst.offset, src.offset, n, W.DT_FLOAT, W.RED_SUM)
        else:
            ref.qsum_reduce(team, dst.offset, src.offset, sc.offset, kind, n)
    assert first_diff(got1, ref.mem) is None
    h.partitions().copy_(torch.from_numpy(init.reshape(world, H)).cuda())
    b.launch()              # graph replay: counters were reset by the last CTA
    b.launch()
    torch.cuda.synchronize()
    assert first_diff(download(h), ref.mem) is None
    tune = b.autotune()
    assert tune.tile_elems in (2048, 4096, 8192, 32768, 131072) and tune.deep in (0, 1)
    h.partitions().copy_(torch.from_numpy(init.reshape(world, H)).cuda())
    b.launch()
    torch.cuda.synchronize()
    assert first_diff(download(h), ref.mem) is None
    # the deep kernel (2 CTAs per SM, 16 quantised members loaded ahead) on the same plan
    for tile in (4096, 8192):
        bd = sg.Batch(descs, sg.Tune(tile, 0, 0, 1))
        h.partitions().copy_(torch.from_numpy(init.reshape(world, H)).cuda())
        bd.launch()
        torch.cuda.synchronize()
        assert first_diff(download(h), ref.mem) is None, tile
        bd.destroy()
    b.destroy()
