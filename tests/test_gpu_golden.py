"""The hand-derived binary32 tree sums of tests/golden/fp32_tree_sum.txt through every GPU
float sum path: the host-issued reduction (k_reduce, tree unrolled in 32-rank blocks), a
device script's reduction (the interpreter) and the batched engine (8-rank blocks with a
carry stack).  Each evaluates the rank-pairwise tree as sums of aligned power-of-two
blocks, and each must land on the values derived by hand from the level-by-level
definition."""
import os

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fp32_tree_sum.txt")


def _cases():
    out = []
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            vals, tree, _seq = [c.strip() for c in line.split(";")]
            out.append((np.array([float(x) for x in vals.split(",")], np.float32), np.float32(float(tree))))
    return out


@pytest.mark.parametrize("path", ["host", "script", "batch"])
def test_fp32_tree_golden_on_every_gpu_path(sg, path):
    cases = _cases()
    assert len(cases) >= 6
    for vals, want in cases:
        P = len(vals)
        h = sg.Heap(P, 4096)   # one heap at a time: each case closes its own
        try:
            _check(sg, h, P, vals, want, path)
        finally:
            h.close()


def _check(sg, h, P, vals, want, path):
    for r in range(P):
        h.view(0, r, torch.float32, 4).copy_(torch.tensor([vals[r], 0, 0, 0], dtype=torch.float32))
    torch.cuda.synchronize()
    sg.clear_status()
    if path == "host":
        sg.reduce(sg.TEAM_WORLD, h.base + 1024, h.base, 1, sg.FLOAT, sg.SUM)
        sg.quiet()
    elif path == "script":
        op = np.zeros((), dtype=W.OP_DTYPE)
        op["kind"], op["dtype"], op["sub"], op["team"] = W.OP_REDUCE, W.DT_FLOAT, W.RED_SUM, 0
        op["issuer"], op["dst"], op["src"], op["n"] = -1, 1024, 0, 1
        ops = np.array([op], dtype=W.OP_DTYPE)
        sg.run_script(torch.from_numpy(ops.view(np.uint8).copy()).cuda(), 1, None)
    else:
        b = sg.Batch([sg.CollDesc(0, P, sg.FLOAT, -1, 1, h.base + 1024, h.base, None)], sg.Tune(2048, 0, 0, 0))
        b.launch()
        torch.cuda.synchronize()
        b.destroy()
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    for r in (0, P - 1):
        got = h.view(1024, r, torch.float32, 1).cpu().numpy()[0]
        assert np.float32(got).view(np.uint32) == want.view(np.uint32), (path, vals.tolist(), float(got), float(want))


def _neumaier_cases():
    out = []
    for line in open(os.path.join(os.path.dirname(GOLD), "neumaier.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            vals, want, _naive = [c.strip() for c in line.split(";")]
            v = np.array([float(x) for x in vals.split(",")], np.float32)
            if np.all((v.view(np.uint32) & 0xFFFF) == 0):   # exact in bfloat16
                out.append((v, np.float32(float(want))))
    return out


@pytest.mark.parametrize("path", ["qsum", "batch"])
def test_neumaier_golden_on_the_quantised_gpu_paths(sg, path):
    """The hand-traced Neumaier sums of tests/golden/neumaier.txt whose values are exact
    in bfloat16, as bf16 codes with scale 1 (the dequantised values are the traced ones):
    the standalone quantised reduce and the batched engine accumulate them in team-rank
    order and must give the traced results bitwise."""
    cases = _neumaier_cases()
    assert len(cases) >= 3
    for vals, want in cases:
        P = len(vals)
        h = sg.Heap(P, 4096)
        try:
            codes = (vals.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)
            for r in range(P):
                h.view(0, r, torch.int16, 8).copy_(torch.tensor([codes[r]] + [0] * 7, dtype=torch.int16))
                h.view(256, r, torch.float32, 4).copy_(torch.tensor([1.0, 0, 0, 0], dtype=torch.float32))
            torch.cuda.synchronize()
            sg.clear_status()
            if path == "qsum":
                sg.qsum_reduce(sg.TEAM_WORLD, h.base + 1024, h.base, h.base + 256, sg.FMT_BF16, 1)
                sg.quiet()
            else:
                b = sg.Batch([sg.CollDesc(0, P, sg.FLOAT, sg.FMT_BF16, 1, h.base + 1024, h.base, h.base + 256)],
                             sg.Tune(2048, 0, 0, 0))
                b.launch()
                torch.cuda.synchronize()
                b.destroy()
            torch.cuda.synchronize()
            assert sg.get_status()[0] == 0
            for r in (0, P - 1):
                got = h.view(1024, r, torch.float32, 1).cpu().numpy()[0]
                assert np.float32(got).view(np.uint32) == want.view(np.uint32), (path, vals.tolist(), float(got))
        finally:
            h.close()


def _golden_rows(name):
    rows = []
    for line in open(os.path.join(os.path.dirname(GOLD), name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([c.strip() for c in line.split(";")])
    return rows


def _quantize_codes(sg, vals, fmt, pin):
    """Codes the GPU quantiser gives `vals` when every 128-element block also holds `pin`
    as its largest magnitude (so the block's scale is exactly 1 for E4M3 pin 448, or for
    bf16 pin 1)."""
    per = 127
    nb = (len(vals) + per - 1) // per
    x = np.zeros((nb, 128), np.float32)
    x[:, 0] = pin
    flat = np.zeros(nb * per, np.float32)
    flat[:len(vals)] = vals
    x[:, 1:] = flat.reshape(nb, per)
    n = nb * 128
    h = sg.Heap(1, 1 << 20)
    try:
        h.view(0, 0, torch.float32, n).copy_(torch.from_numpy(x.reshape(-1)))
        qb = 1 if fmt == sg.FMT_E4M3 else 2
        q_off, s_off = 1 << 18, 1 << 19
        sg.clear_status()
        sg.quantize(sg.TEAM_WORLD, h.base + q_off, h.base + s_off, h.base, fmt, n)
        sg.quiet()
        assert sg.get_status()[0] == 0
        scales = h.view(s_off, 0, torch.float32, nb).cpu().numpy()
        assert np.all(scales == 1.0)
        dt = torch.uint8 if qb == 1 else torch.int16
        q = h.view(q_off, 0, dt, n).cpu().numpy().reshape(nb, 128)[:, 1:].reshape(-1)[:len(vals)]
        return q.astype(np.uint8) if qb == 1 else q.view(np.uint16)
    finally:
        h.close()


def test_e4m3_encoding_golden_on_the_gpu_quantiser(sg, orc):
    """The golden encodings up to 448, every finite code's value (round trip) and every
    midpoint of adjacent codes (ties to the even code), through the GPU quantiser with
    scale 1."""
    vals, want = [], []
    for row in _golden_rows("e4m3.txt"):
        # (magnitudes above 448 saturate: they would set the block's scale, so they stay
        # with the oracle's pin and the GPU parity tests)
        if row[0].startswith("enc") and abs(float(row[0][3:])) <= 448.0:
            vals.append(float(row[0][3:]))
            want.append(int(row[1], 16))
    dec = [orc.e4m3_decode(c) for c in range(0x7F)]
    for c in range(0x7F):
        vals += [dec[c], -dec[c]]
        want += [c, c | 0x80 if c else 0x80]
    for c in range(0x7E):
        vals.append((dec[c] + dec[c + 1]) / 2)
        want.append(c if c % 2 == 0 else c + 1)
    got = _quantize_codes(sg, np.array(vals, np.float32), sg.FMT_E4M3, 448.0)
    bad = [(v, int(g), w) for v, g, w in zip(vals, got, want) if int(g) != w]
    assert not bad, bad[:8]


def test_bf16_encoding_golden_on_the_gpu_quantiser(sg, orc):
    """The golden bf16 encodings of magnitude at most 1 and the midpoints of adjacent bf16
    values in [1/256, 1) (ties to even), through the GPU quantiser with scale 1."""
    vals, want = [], []
    for v, code in _golden_rows("bf16.txt"):
        if abs(float(v)) <= 1.0:
            vals.append(float(v))
            want.append(int(code, 16))
    for c in range(0x3B80, 0x3F80, 3):   # 2^-8 <= value < 1
        lo, hi = orc.bf16_decode(c), orc.bf16_decode(c + 1)
        vals.append((lo + hi) / 2)
        want.append(c if c % 2 == 0 else c + 1)
    assert len(vals) > 300
    got = _quantize_codes(sg, np.array(vals, np.float32), sg.FMT_BF16, 1.0)
    bad = [(v, int(g), w) for v, g, w in zip(vals, got, want) if int(g) != w]
    assert not bad, bad[:8]


def test_gpu_quantiser_divides_exactly(sg):
    """The hand-derived bf16 tie of the oracle's quantiser pin: in a block of largest
    magnitude 7, x = 4.716796875 gives x / 7 = 345/512 exactly, halfway between 0x3F2C
    (even) and 0x3F2D; only a correctly rounded quotient (not x times a rounded 1/7)
    reaches the tie and its even code."""
    h = sg.Heap(1, 1 << 16)
    try:
        x = np.zeros(128, np.float32)
        x[0], x[1] = 7.0, 4.716796875
        h.view(0, 0, torch.float32, 128).copy_(torch.from_numpy(x))
        sg.clear_status()
        sg.quantize(sg.TEAM_WORLD, h.base + 4096, h.base + 8192, h.base, sg.FMT_BF16, 128)
        sg.quiet()
        assert sg.get_status()[0] == 0
        assert h.view(8192, 0, torch.float32, 1).cpu().numpy()[0] == 7.0
        assert int(h.view(4096, 0, torch.int16, 2).cpu().numpy().view(np.uint16)[1]) == 0x3F2C
    finally:
        h.close()
