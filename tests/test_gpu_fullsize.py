"""Full-size parity of the benchmark's own workload (64 PEs x 768 MiB, PEs = clusters of
2 CTAs, the launch configuration bench.py times): the largest point of every op family
runs once and sampled outputs are compared with the oracle applied to the sampled
inputs (a small heap holding only the sampled positions)."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

MiB = 1 << 20
NS = 2048  # sampled positions per op


@pytest.fixture(scope="module")
def step(sg):
    import bench

    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = bench.GpuStep(torch, sg, s)
    yield bench, g, s
    g.heap.close()


def _gather(parts, pes, offs, width):
    """bytes [off, off+width) of each PE in pes at each offset -> numpy [len(pes), len(offs), width]"""
    idx = torch.as_tensor(offs, dtype=torch.int64, device="cuda")[:, None] + torch.arange(width, device="cuda")[None, :]
    rows = parts[torch.as_tensor(pes, device="cuda")]
    return rows[:, idx.reshape(-1)].reshape(len(pes), len(offs), width).cpu().numpy()


def _run(bench, g, s, name, fam, m):
    g.run_point(name, fam, m)
    s.synchronize()


@pytest.mark.parametrize("kind", ["put", "get"])
def test_ring_256MiB(sg, orc, step, kind):
    bench, g, s = step
    m = 256 * MiB
    _run(bench, g, s, f"{kind}_nbi_ring", kind, m)
    assert sg.get_status()[0] == 0
    parts = g.heap.partitions()
    rng = np.random.default_rng(7)
    offs = np.sort(rng.choice(m // 16, NS, replace=False)) * 16
    P = bench.NPES
    a = _gather(parts, list(range(P)), bench.A_OFF + offs, 16)
    b = _gather(parts, list(range(P)), bench.B_OFF + offs, 16)
    # oracle on a heap holding only the samples: A at [0, NS*16), B at [NS*16, 2*NS*16)
    w = NS * 16
    ref = orc.Heap(P, 2 * w)
    for p in range(P):
        ref.pe(p)[:w] = a[p].reshape(-1)
    for p in range(P):
        q = (p + 1) % P
        if kind == "put":
            ref.put(w, 0, w, q, p)
        else:
            ref.get(w, 0, w, q, p)
    for p in range(P):
        assert np.array_equal(b[p].reshape(-1), ref.pe(p)[w:]), p


@pytest.mark.parametrize("dt,op,n", [("int32", "sum", 1 << 24), ("int64", "sum", 1 << 24), ("int32", "max", 1 << 24),
                                     ("int64", "max", 1 << 24), ("int32", "sum", 1 << 20), ("int64", "max", 1 << 20),
                                     ("int32", "max", 1 << 22)])
def test_reduce_full_points(sg, orc, step, dt, op, n):
    """The largest reduce points (16 Mi elements: the one-vector-per-thread kernel) and the
    1 Mi / 4 Mi points the bulk ring runs (4-16 MiB per member)."""
    bench, g, s = step
    _run(bench, g, s, f"reduce_{dt}_{op}", "reduce", n)
    parts = g.heap.partitions()
    es = 4 if dt == "int32" else 8
    src = bench.A_OFF + (bench.I32_OFF if dt == "int32" else 0)
    k = np.sort(np.random.default_rng(3).choice(n, NS, replace=False))
    P = bench.NPES
    x = _gather(parts, list(range(P)), src + k * es, es)
    y = _gather(parts, [0, 17, P - 1], bench.B_OFF + k * es, es)
    ref = orc.Heap(P, 2 * NS * es)
    for p in range(P):
        ref.pe(p)[:NS * es] = x[p].reshape(-1)
    ref.reduce((0, 1, P), NS * es, 0, NS, W.DT_INT32 if dt == "int32" else W.DT_INT64,
               W.RED_SUM if op == "sum" else W.RED_MAX)
    for i, p in enumerate([0, 17, P - 1]):
        assert np.array_equal(y[i].reshape(-1), ref.pe(p)[NS * es:])


def test_broadcast_256MiB(sg, orc, step):
    bench, g, s = step
    m = 256 * MiB
    _run(bench, g, s, "broadcast", "broadcast", m)
    parts = g.heap.partitions()
    offs = np.sort(np.random.default_rng(5).choice(m // 16, NS, replace=False)) * 16
    P = bench.NPES
    a = _gather(parts, list(range(P)), bench.A_OFF + offs, 16)
    b = _gather(parts, list(range(P)), bench.B_OFF + offs, 16)
    w = NS * 16
    ref = orc.Heap(P, 2 * w)
    for p in range(P):
        ref.pe(p)[:w] = a[p].reshape(-1)
    ref.broadcast((0, 1, P), w, 0, w, P - 1)
    for p in range(P):
        assert np.array_equal(b[p].reshape(-1), ref.pe(p)[w:])


def test_alltoall_1MiB_per_pair(sg, orc, step):
    bench, g, s = step
    m = 1 * MiB
    _run(bench, g, s, "alltoall", "alltoall", m)
    parts = g.heap.partitions()
    P = bench.NPES
    # samples: (source PE i, destination PE j, byte offset t inside the block)
    rng = np.random.default_rng(9)
    t = rng.choice(m // 16, 64, replace=False) * 16
    src = _gather(parts, list(range(P)), bench.A_OFF + (np.arange(P)[:, None] * m + t[None, :]).reshape(-1), 16)
    dst = _gather(parts, list(range(P)), bench.B_OFF + (np.arange(P)[:, None] * m + t[None, :]).reshape(-1), 16)
    # oracle heap with blocks of 64 samples x 16 bytes
    bw = 64 * 16
    ref = orc.Heap(P, 2 * P * bw)
    for p in range(P):
        ref.pe(p)[:P * bw] = src[p].reshape(-1)
    ref.alltoall((0, 1, P), P * bw, 0, bw)
    for p in range(P):
        assert np.array_equal(dst[p].reshape(-1), ref.pe(p)[P * bw:])


@pytest.mark.parametrize("dt", ["int32", "int64"])
def test_fcollect_16Mi_total(sg, orc, step, dt):
    bench, g, s = step
    es = 4 if dt == "int32" else 8
    P = bench.NPES
    n = (1 << 24) // P
    _run(bench, g, s, f"fcollect_{dt}", "fcollect", n)
    parts = g.heap.partitions()
    src = bench.A_OFF + (bench.I32_OFF if dt == "int32" else 0)
    k = np.sort(np.random.default_rng(11).choice(n, 256, replace=False))
    x = _gather(parts, list(range(P)), src + k * es, es)                      # [P, 256, es]
    dpos = (np.arange(P)[:, None] * n + k[None, :]).reshape(-1) * es          # block r, element k
    y = _gather(parts, [0, P // 2], bench.B_OFF + dpos, es)
    ref = orc.Heap(P, 256 * es + P * 256 * es)
    for p in range(P):
        ref.pe(p)[:256 * es] = x[p].reshape(-1)
    ref.fcollect((0, 1, P), 256 * es, 0, 256 * es)
    for i, p in enumerate([0, P // 2]):
        assert np.array_equal(y[i].reshape(-1), ref.pe(p)[256 * es:])
