"""Pins of the CPU oracle to facts fixed by the mathematics and the paper's model,
independent of the oracle's own code: hand-computed fixtures (tests/golden), closed
forms, brute force on tiny inputs, invariants and published generator outputs."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([c.strip() for c in line.split(";")])
    return rows


# ----------------------------------------------------------------- generators
def test_splitmix64_published_outputs(orc):
    # first three outputs of splitmix64 seeded with 0 (Vigna's reference splitmix64.c)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = W.SplitMix64(0)
    assert [r.next() for _ in range(3)] == want
    assert orc.cb64(0, 0) == want[0]
    # cb64(s, i) is the first output of the stream seeded with s ^ i
    for s, i in [(5, 9), (W.MASTER_SEED, 123456789), (2**64 - 1, 3)]:
        assert orc.cb64(s, i) == W.SplitMix64(s ^ i).next() == W.cb64(s, i)
    idx = np.arange(1000, dtype=np.uint64)
    assert np.array_equal(W.cb64_np(77, idx), np.array([orc.cb64(77, int(i)) for i in idx], np.uint64))


def test_staged_payload_word_layout():
    """Staged payload words follow the request record's definition: four words per
    SplitMix64 draw of (seed, PE, word // 4), word q taking bytes 7 - 2q (high bfloat16) and
    6 - 2q (low) of the draw, each byte k coded as the bfloat16 of
    (-1)^(k >> 7) * (1 + (k & 127) / 128) -- checked word by word from the published first
    output and from the bytes' values."""
    seed, pe = 0x1234567, 5
    w = W.serve_payload_words(seed, pe, 0, 4 * 7 + 3)
    for j in range(len(w)):
        z = W.SplitMix64(seed ^ ((pe << 40) | (j // 4))).next()
        hi, lo = (z >> (56 - 16 * (j % 4))) & 255, (z >> (48 - 16 * (j % 4))) & 255
        for k, half in ((hi, int(w[j]) >> 16), (lo, int(w[j]) & 0xFFFF)):
            v = np.array([half << 16], np.uint32).view(np.float32)[0]   # the bfloat16 as binary32
            assert v == (-1.0 if k >> 7 else 1.0) * (1 + (k & 127) / 128.0), (j, k, half)
    # an offset start gives the same words (word j's draw depends on j alone)
    assert np.array_equal(W.serve_payload_words(seed, pe, 6, 20), w[6:26])


def test_torch_generator_matches_numpy():
    torch = pytest.importorskip("torch")
    idx = np.arange(5000, dtype=np.int64) * 7919
    a = W.cb64_torch(1234567, torch.from_numpy(idx)).numpy().view(np.uint64)
    assert np.array_equal(a, W.cb64_np(1234567, idx.astype(np.uint64)))
    b = W.uniform_ints_torch(99, torch.from_numpy(idx), -(1 << 20), 1 << 20).numpy()
    assert np.array_equal(b, W.uniform_ints_np(99, idx.astype(np.uint64), -(1 << 20), 1 << 20))


# ----------------------------------------------------------------- RMA
def test_put_get_round_trip_and_untouched_bytes(orc):
    npes, H = 3, 4096
    init = np.random.default_rng(1).integers(0, 256, npes * H, dtype=np.uint8)
    h = orc.Heap(npes, H, init)
    h.put(dst=1000, src=8, nbytes=777, pe=2, issuer=0)          # PE0[8:785] -> PE2[1000:1777]
    h.get(dst=2000, src=1000, nbytes=777, pe=2, issuer=1)       # PE2[1000:..] -> PE1[2000:..]
    want = init.copy().reshape(npes, H)
    want[2, 1000:1777] = init.reshape(npes, H)[0, 8:785]
    want[1, 2000:2777] = init.reshape(npes, H)[0, 8:785]
    assert np.array_equal(h.mem.reshape(npes, H), want)


def test_rma_range_errors(orc):
    h = orc.Heap(2, 256)
    with pytest.raises(orc.OracleError):
        h.put(dst=250, src=0, nbytes=8, pe=1, issuer=0)
    with pytest.raises(orc.OracleError):
        h.put(dst=0, src=0, nbytes=8, pe=2, issuer=0)


# ----------------------------------------------------------------- AMOs
def test_fetch_add_increments_invariant(orc):
    h = orc.Heap(2, 64)
    rng = W.SplitMix64(3)
    vals = [rng.randint(1, 1 << 20) for _ in range(200)]
    fetched = [h.amo64(W.OP_FADD, 1, 16, v) for v in vals]
    assert fetched == list(np.cumsum([0] + vals[:-1]))
    assert h.view(1, 16, 1, np.int64)[0] == sum(vals)


def test_amo_wraparound_cswap_xor(orc):
    h = orc.Heap(1, 64)
    h.view(0, 0, 1, np.int64)[0] = 2**63 - 1
    assert h.amo64(W.OP_FADD, 0, 0, 1) == 2**63 - 1
    assert h.view(0, 0, 1, np.int64)[0] == -(2**63)
    # compare_swap: stores only on equality, returns the old value either way
    assert h.amo64(W.OP_CSWAP, 0, 0, 5, cond=7) == -(2**63)
    assert h.view(0, 0, 1, np.int64)[0] == -(2**63)
    assert h.amo64(W.OP_CSWAP, 0, 0, 5, cond=-(2**63)) == -(2**63)
    assert h.view(0, 0, 1, np.int64)[0] == 5
    # fetch_xor twice with the same operand restores the word
    h.amo64(W.OP_FXOR, 0, 0, 0x0F0F)
    assert h.view(0, 0, 1, np.int64)[0] == 5 ^ 0x0F0F
    h.amo64(W.OP_FXOR, 0, 0, 0x0F0F)
    assert h.view(0, 0, 1, np.int64)[0] == 5
    # int32 flavour wraps at 2^31
    h.view(0, 8, 1, np.int32)[0] = 2**31 - 1
    assert h.amo32(W.OP_FADD, 0, 8, 2) == 2**31 - 1
    assert h.view(0, 8, 1, np.int32)[0] == -(2**31) + 1


def test_signal_ops(orc):
    h = orc.Heap(2, 128)
    h.view(0, 0, 4, np.uint8)[:] = [1, 2, 3, 4]
    h.put_signal(dst=32, src=0, nbytes=4, sig=64, sig_op=W.SIG_ADD, v=3, pe=1, issuer=0)
    h.put_signal(dst=40, src=0, nbytes=4, sig=64, sig_op=W.SIG_ADD, v=2**64 - 1, pe=1, issuer=0)
    assert list(h.view(1, 32, 4, np.uint8)) == [1, 2, 3, 4]
    assert h.view(1, 64, 1, np.uint64)[0] == 2  # 3 + (2^64 - 1) wraps to 2
    assert h.signal_test(1, 64, W.CMP_EQ, 2) and h.signal_test(1, 64, W.CMP_GE, 2)
    assert not h.signal_test(1, 64, W.CMP_GT, 2) and h.signal_test(1, 64, W.CMP_LT, 3)
    h.put_signal(dst=32, src=0, nbytes=0, sig=64, sig_op=W.SIG_SET, v=9, pe=1, issuer=0)
    assert h.view(1, 64, 1, np.uint64)[0] == 9 and h.signal_test(1, 64, W.CMP_NE, 2)


# ----------------------------------------------------------------- collectives
def _tagged(npes, H):
    """Every byte tagged by (pe, offset) so any misplaced byte is visible."""
    a = np.zeros((npes, H), np.uint8)
    for p in range(npes):
        a[p] = (np.arange(H) * 7 + p * 31) % 251
    return a.reshape(-1)


def test_broadcast_definition_root_included(orc):
    npes, H = 5, 1024
    init = _tagged(npes, H)
    h = orc.Heap(npes, H, init)
    team = (1, 1, 4)  # PEs 1..4, root = team rank 2 = PE 3
    h.broadcast(team, dst=512, src=0, nbytes=100, root=2)
    want = init.reshape(npes, H).copy()
    for p in (1, 2, 3, 4):
        want[p, 512:612] = init.reshape(npes, H)[3, 0:100]
    assert np.array_equal(h.mem.reshape(npes, H), want)


def test_fcollect_definition(orc):
    npes, H = 4, 512
    init = _tagged(npes, H)
    h = orc.Heap(npes, H, init)
    team = (0, 2, 2)  # PEs 0 and 2
    h.fcollect(team, dst=256, src=0, nbytes=40)
    ref = init.reshape(npes, H)
    for p in (0, 2):
        assert np.array_equal(h.pe(p)[256:296], ref[0, 0:40])
        assert np.array_equal(h.pe(p)[296:336], ref[2, 0:40])
    assert np.array_equal(h.pe(1), ref[1]) and np.array_equal(h.pe(3), ref[3])


def test_alltoall_is_exact_transpose_permutation(orc):
    P, m = 5, 24
    H = 2 * P * m
    h = orc.Heap(P, H)
    # src block j of PE i holds the tag (i, j) in every 8-byte word
    for i in range(P):
        for j in range(P):
            h.view(i, j * m, m // 8, np.int64)[:] = 1000 * i + j
    h.alltoall((0, 1, P), dst=P * m, src=0, m=m)
    seen = []
    for j in range(P):
        for i in range(P):
            blk = h.view(j, P * m + i * m, m // 8, np.int64)
            assert np.all(blk == blk[0])
            seen.append(int(blk[0]))
            assert blk[0] == 1000 * i + j          # dst block i of PE j = src block j of PE i
    assert sorted(seen) == sorted(1000 * i + j for i in range(P) for j in range(P))


@pytest.mark.parametrize("dtype,npdt,bits", [(W.DT_INT32, np.int32, 32), (W.DT_INT64, np.int64, 64)])
def test_int_reduce_brute_force_tiny(orc, dtype, npdt, bits):
    rng = np.random.default_rng(bits)
    for P in (1, 2, 3, 4):
        for n in (1, 5, 8):
            H = 2 * n * 8
            h = orc.Heap(P, H)
            lim = 2 ** (bits - 1)
            data = rng.integers(-lim, lim, (P, n), dtype=np.int64).astype(npdt)
            for r in range(P):
                h.view(r, 0, n, npdt)[:] = data[r]
            for op in (W.RED_SUM, W.RED_MAX, W.RED_MIN):
                h.reduce((0, 1, P), dst=n * 8, src=0, nelems=n, dtype=dtype, op=op)
                for k in range(n):
                    col = [int(data[r, k]) for r in range(P)]
                    if op == W.RED_SUM:
                        e = sum(col) % (1 << bits)
                        e = e - (1 << bits) if e >= lim else e
                    else:
                        e = max(col) if op == W.RED_MAX else min(col)
                    for r in range(P):
                        assert int(h.view(r, n * 8, n, npdt)[k]) == e


def test_reduce_closed_form_and_one_hot(orc):
    P, n = 7, 300
    h = orc.Heap(P, 8 * n * 2)
    for r in range(P):
        h.view(r, 0, n, np.int64)[:] = r + np.arange(n)
    h.reduce((0, 1, P), dst=8 * n, src=0, nelems=n, dtype=W.DT_INT64, op=W.RED_SUM)
    k = np.arange(n)
    for r in range(P):
        assert np.array_equal(h.view(r, 8 * n, n, np.int64), P * k + P * (P - 1) // 2)
    # one-hot: max picks the hot rank's value, min picks zero
    for r in range(P):
        h.view(r, 0, n, np.float32)[:] = np.where(k % P == r, 1.5 + r, 0.0)
    h.reduce((0, 1, P), dst=4 * n, src=0, nelems=n, dtype=W.DT_FLOAT, op=W.RED_MAX)
    assert np.array_equal(h.view(3, 4 * n, n, np.float32), (1.5 + k % P).astype(np.float32))
    h.reduce((0, 1, P), dst=4 * n, src=0, nelems=n, dtype=W.DT_FLOAT, op=W.RED_MIN)
    assert np.all(h.view(0, 4 * n, n, np.float32) == 0.0)


def test_reduce_in_place(orc):
    P, n = 3, 10
    h = orc.Heap(P, 8 * n)
    for r in range(P):
        h.view(r, 0, n, np.int64)[:] = 10 ** r
    h.reduce((0, 1, P), dst=0, src=0, nelems=n, dtype=W.DT_INT64, op=W.RED_SUM)
    for r in range(P):
        assert np.all(h.view(r, 0, n, np.int64) == 111)


def test_fp32_tree_golden(orc):
    for vals, tree, seq in _golden("fp32_tree_sum.txt"):
        v = [float(x) for x in vals.split(",")]
        assert orc.tree_sum_f32(v) == np.float32(float(tree)), vals
        # the same values through the team reduce of the heap model
        P = len(v)
        h = orc.Heap(P, 8)
        for r in range(P):
            h.view(r, 0, 1, np.float32)[0] = v[r]
        h.reduce((0, 1, P), dst=4, src=0, nelems=1, dtype=W.DT_FLOAT, op=W.RED_SUM)
        assert h.view(P - 1, 4, 1, np.float32)[0] == np.float32(float(tree))
        s = np.float32(0)
        for x in v:
            s = np.float32(s + np.float32(x))
        assert s == np.float32(float(seq))


def test_fp32_tree_within_pairwise_bound(orc):
    # |tree - exact| <= ceil(log2 P) * u * sum|x| / (1 - ceil(log2 P) u)  (Higham,
    # Accuracy and Stability of Numerical Algorithms, Sec. 4.2), checked against exact
    # rational sums of the binary32 inputs; the 1e-6 gate follows for P <= 128.
    rng = W.SplitMix64(11)
    u = 2.0 ** -24
    for P in (2, 3, 7, 64, 100, 128):
        for _ in range(20):
            v = [np.float32(rng.normal() * 10 ** rng.randint(-3, 3)) for _ in range(P)]
            exact = sum(Fraction(float(x)) for x in v)
            absum = sum(abs(Fraction(float(x))) for x in v)
            got = Fraction(float(orc.tree_sum_f32(v)))
            L = math.ceil(math.log2(P))
            assert abs(got - exact) <= Fraction(L * u / (1 - L * u)) * absum
            assert abs(got - exact) <= Fraction(1, 10 ** 6) * absum


# ----------------------------------------------------------------- codecs
def test_e4m3_golden_and_exhaustive(orc):
    for row in _golden("e4m3.txt"):
        if row[0].startswith("enc"):
            assert orc.e4m3_encode(float(row[0][3:])) == int(row[1], 16), row
        else:
            v = orc.e4m3_decode(int(row[0], 16))
            if row[1] == "nan":
                assert math.isnan(v)
            else:
                assert v == float(row[1]) and math.copysign(1, v) == math.copysign(1, float(row[1]))
    vals = [orc.e4m3_decode(c) for c in range(0x7F)]
    assert all(b > a for a, b in zip(vals, vals[1:]))           # monotone: codes 0..126
    for c in list(range(0x7F)) + list(range(0x80, 0xFF)):
        assert orc.e4m3_encode(orc.e4m3_decode(c)) == c         # every finite code round trips
    # every midpoint between adjacent codes goes to the even code
    for c in range(0x7E):
        mid = (vals[c] + vals[c + 1]) / 2
        assert orc.e4m3_encode(mid) == (c if c % 2 == 0 else c + 1)


def test_bf16_golden_and_round_trip(orc):
    for v, code in _golden("bf16.txt"):
        assert orc.bf16_encode(float(v)) == int(code, 16), v
    for c in range(0, 0x10000, 37):
        if (c & 0x7F80) == 0x7F80:
            continue  # inf / nan
        assert orc.bf16_encode(orc.bf16_decode(c)) == c


def test_neumaier_golden_and_exact_rational(orc):
    for vals, want, naive in _golden("neumaier.txt"):
        v = [float(x) for x in vals.split(",")]
        assert orc.neumaier_f32(v) == np.float32(float(want))
        s = np.float32(0)
        for x in v:
            s = np.float32(s + np.float32(x))
        assert s == np.float32(float(naive))
    # error vs the exact rational sum stays within 2u|y| + 2P^2 u^2 sum|x| (Neumaier's
    # bound) on random tiny inputs
    rng = W.SplitMix64(5)
    u = 2.0 ** -24
    for P in (2, 3, 5, 16, 128):
        for _ in range(30):
            v = [np.float32(rng.normal() * 2.0 ** rng.randint(-20, 20)) for _ in range(P)]
            exact = sum(Fraction(float(x)) for x in v)
            absum = sum(abs(Fraction(float(x))) for x in v)
            got = Fraction(float(orc.neumaier_f32(v)))
            assert abs(got - exact) <= Fraction(2 * u) * abs(exact) + Fraction(2 * P * P * u * u) * absum


def test_quantize_scales_and_codes(orc):
    # block of 128 with amax 448: s = 448/448 = 1 and representable values encode exactly
    x = np.array([(-1) ** i * [448, 1, 1.5, 0.015625, 2.0 ** -9, 0][i % 6] for i in range(128)],
                 np.float32)
    q, s = orc.quantize(x, W.FMT_E4M3)
    assert s.tolist() == [1.0]
    assert [orc.e4m3_decode(int(c)) for c in q] == [float(t) for t in x]
    # bf16: s = amax; x / s in [-1, 1]; a ragged last block gets its own scale; an all-zero
    # block gets s = 1
    x = np.concatenate([np.full(128, 0.0), np.array([2.0, -4.0, 1.0], np.float32)]).astype(np.float32)
    q, s = orc.quantize(x, W.FMT_BF16)
    assert s.tolist() == [1.0, 4.0]
    assert [orc.bf16_decode(int(c)) for c in q[128:]] == [0.5, -1.0, 0.25]
    assert np.all(q[:128] == 0)
    # a tie that only the exact quotient reaches: s = 7, x = 4.716796875, x / s = 345/512 =
    # 0.673828125 exactly, halfway between bf16 0.671875 (0x3F2C, even) and 0.67578125
    # (0x3F2D); x times a rounded 1/7 lands above the midpoint instead
    q, s = orc.quantize(np.array([7.0, 4.716796875], np.float32), W.FMT_BF16)
    assert s.tolist() == [7.0] and int(q[1]) == 0x3F2C


def test_qsum_single_member_is_dequantised_input(orc):
    n = 300
    x = (W.normals_np(9, n) * 3).astype(np.float32)
    for fmt in (W.FMT_BF16, W.FMT_E4M3):
        q, s = orc.quantize(x, fmt)
        qs = 1 if fmt == W.FMT_E4M3 else 2
        H = 4096
        h = orc.Heap(2, H)
        h.pe(1)[0:n * qs] = q.view(np.uint8)
        h.pe(1)[2048:2048 + 4 * len(s)] = s.view(np.uint8)
        h.qsum_reduce((1, 1, 1), dst=1024, q_off=0, s_off=2048, fmt=fmt, n=n)
        dec = np.array([(orc.e4m3_decode(int(c)) if fmt else orc.bf16_decode(int(c))) for c in q])
        want = (dec.astype(np.float32) * np.repeat(s, 128)[:n]).astype(np.float32)
        assert np.array_equal(h.view(1, 1024, n, np.float32), want)
        # quantisation error bound per element: half a unit in the last place of the code
        # times the scale (e4m3: 2^-4 relative, plus the subnormal step 2^-9 * s)
        rel = 2.0 ** -4 if fmt else 2.0 ** -8
        sub = 2.0 ** -10 if fmt else 0.0
        sc = np.repeat(s, 128)[:n].astype(np.float64)
        assert np.all(np.abs(want - x) <= rel * np.abs(x) + sub * sc * 1.0001 + 1e-30)


# ----------------------------------------------------------------- serialisation checker
def _replay_ok(ops, w0, fetched, final):
    for perm in itertools.permutations(range(len(ops))):
        cur, ok = w0, True
        for j in perm:
            k, v, c = ops[j]
            if fetched[j] != cur:
                ok = False
                break
            if k == W.OP_FADD:
                cur = (cur + v + 2**63) % 2**64 - 2**63
            elif k == W.OP_CSWAP:
                cur = v if cur == c else cur
            else:
                cur = ((cur % 2**64) ^ (v % 2**64) + 2**63) % 2**64 - 2**63
        if ok and (final is None or cur == final):
            return True
    return False


def test_serialisation_checker_vs_brute_force(orc):
    rng = W.SplitMix64(17)
    agree = {True: 0, False: 0}
    for trial in range(400):
        m = rng.randint(1, 5)
        w0 = rng.randint(0, 3)
        ops = []
        for _ in range(m):
            k = [W.OP_FADD, W.OP_CSWAP, W.OP_FXOR][rng.below(3)]
            ops.append((k, rng.randint(0, 3), rng.randint(0, 3)))
        # a true serial execution in a random order gives valid fetched values ...
        order = list(range(m))
        for i in range(m - 1, 0, -1):
            j = rng.below(i + 1)
            order[i], order[j] = order[j], order[i]
        cur, fetched = w0, [0] * m
        for j in order:
            k, v, c = ops[j]
            fetched[j] = cur
            cur = cur + v if k == W.OP_FADD else (v if (k == W.OP_CSWAP and cur == c) else
                                                  (cur ^ v if k == W.OP_FXOR else cur))
        final = cur
        if trial % 2:   # ... then perturb half of the cases
            fetched[rng.below(m)] += rng.randint(-1, 1)
            final += rng.randint(-1, 1) if rng.below(2) else 0
        want = _replay_ok(ops, w0, fetched, final)
        n = len(ops)
        got = orc.check_serialisation(
            np.zeros(n), [o[0] for o in ops], [o[1] for o in ops], [o[2] for o in ops],
            fetched, np.full(n, w0), np.full(n, final))
        assert (got == 0) == want, (ops, w0, fetched, final)
        agree[want] += 1
    assert agree[True] > 50 and agree[False] > 50


def test_serialisation_checker_groups_and_long_chain(orc):
    # 100k fetch_adds on one word, fetched = a valid serial order shuffled: valid; one
    # fetched value changed: invalid; a second, independent group is checked separately
    n = 100000
    v = (np.arange(n) % 97 + 1).astype(np.int64)
    perm = np.random.default_rng(0).permutation(n)
    fetched = np.zeros(n, np.int64)
    fetched[perm] = np.cumsum(np.concatenate([[0], v[perm][:-1]]))
    kinds = np.full(n, W.OP_FADD)
    g = np.zeros(n, np.int64)
    assert orc.check_serialisation(g, kinds, v, np.zeros(n), fetched, np.zeros(n), np.full(n, v.sum())) == 0
    bad = fetched.copy()
    bad[123] += 1
    assert orc.check_serialisation(g, kinds, v, np.zeros(n), bad, np.zeros(n), None) == 1
    g2 = np.concatenate([g, np.ones(3, np.int64)])
    k2 = np.concatenate([kinds, np.full(3, W.OP_CSWAP)])
    v2 = np.concatenate([v, [9, 8, 7]])
    c2 = np.concatenate([np.zeros(n, np.int64), [5, 5, 9]])
    f2 = np.concatenate([fetched, [5, 9, 9]])   # 5 -> (cswap 5->9) -> 9 ; then two failed/ok
    w02 = np.concatenate([np.zeros(n, np.int64), [5, 5, 5]])
    # group 1: start 5: op0 (c=5,v=9) succeeds -> 9; op1 (c=5) fails at 9; op2 (c=9,v=7) -> 7
    fin = np.concatenate([np.full(n, v.sum()), [7, 7, 7]])
    assert orc.check_serialisation(g2, k2, v2, c2, f2, w02, fin) == 0


# ----------------------------------------------------------------- AMO streams
def test_amo_stream_single_kind_closed_forms(orc):
    nlog = 10
    nw = 1 << nlog
    tseed, oseed = 111, 222
    init = W.cb64_np(tseed, np.arange(nw, dtype=np.uint64)).view(np.int64)
    count = 20000
    r = W.cb64_np(oseed, np.arange(count, dtype=np.uint64))
    # fetch_add only: final = init + sum of (r mod 2^20) + 1 per word (order independent)
    ops = W.amo_stream_np(5, count, nlog, only=W.AMO_CODE_FADD)
    t = init.copy()
    orc.amo_stream(t, ops, oseed, tseed)
    w = (ops & ((1 << 27) - 1)).astype(np.int64)
    inc = ((r % np.uint64(1 << 20)) + np.uint64(1)).astype(np.int64)
    want = init.copy()
    np.add.at(want, w, inc)
    assert np.array_equal(t, want)
    # fetch_xor only: final = init ^ xor of operands per word
    ops = W.amo_stream_np(6, count, nlog, only=W.AMO_CODE_FXOR)
    t = init.copy()
    orc.amo_stream(t, ops, oseed, tseed)
    w = (ops & ((1 << 27) - 1)).astype(np.int64)
    want = init.view(np.uint64).copy()
    np.bitwise_xor.at(want, w, np.where(r == 0, np.uint64(1), r))
    assert np.array_equal(t.view(np.uint64), want)
    # compare_swap only, condition = initial value: the first op on a word succeeds,
    # every later one fails and fetches the first one's value
    ops = W.amo_stream_np(7, count, nlog, only=W.AMO_CODE_CSWAP)
    t = init.copy()
    f = orc.amo_stream(t, ops, oseed, tseed)
    w = (ops & ((1 << 27) - 1)).astype(np.int64)
    first = {}
    for i, ww in enumerate(w):
        if ww not in first:
            first[ww] = i
            assert f[i] == init[ww]
        else:
            assert f[i] == r[first[ww]].view(np.int64)
    for ww, i in first.items():
        assert t[ww] == r[i].view(np.int64)


def test_zipf_generator_shape():
    n = 1 << 27
    ranks = W.zipf_ranks_np(3, 200000, n, 1.1)
    assert ranks.min() >= 1 and ranks.max() <= n
    # P(rank = 1) = 1 / H_{n,s}; H_{2^27,1.1} ~ zeta(1.1) - n^-0.1/0.1 ~ 10.584 - 1.55
    p1 = (ranks == 1).mean()
    assert abs(p1 - 1 / 9.03) < 0.01
    ops = W.amo_stream_np(3, 1000, 27, dist="zipf")
    assert ops.dtype == np.uint32 and np.all((ops >> 27) <= 2)


# ----------------------------------------------------------------- scripts
def test_script_dispatch_matches_single_ops(orc):
    npes, H = 3, 2048
    init = _tagged(npes, H)
    ops = np.zeros(6, W.OP_DTYPE)
    ops[0] = (W.OP_PUT, 0, 0, 0, 2, 0, 100, 0, 64, 0, 0, 0)
    ops[1] = (W.OP_GET, 0, 0, 0, 2, 1, 300, 100, 64, 0, 0, 0)
    ops[2] = (W.OP_FADD, W.DT_INT64, 0, 0, 1, 0, 512, 0, 0, 5, 0, 0)
    ops[3] = (W.OP_CSWAP, W.DT_INT64, 0, 0, 1, 2, 512, 0, 0, 9, 0, 0)
    ops[4] = (W.OP_REDUCE, W.DT_INT32, W.RED_MAX, 0, 0, -1, 1024, 0, 16, 0, 0, 0)
    ops[5] = (W.OP_BCAST, 0, 0, 0, 1, -1, 1536, 1024, 64, 0, 0, 0)
    a = orc.Heap(npes, H, init)
    f = a.run_script(ops)
    b = orc.Heap(npes, H, init)
    b.put(100, 0, 64, pe=2, issuer=0)
    b.get(300, 100, 64, pe=2, issuer=1)
    f2 = b.amo64(W.OP_FADD, 1, 512, 5)
    f3 = b.amo64(W.OP_CSWAP, 1, 512, 9, 0)
    b.reduce((0, 1, npes), 1024, 0, 16, W.DT_INT32, W.RED_MAX)
    b.broadcast((0, 1, npes), 1536, 1024, 64, 1)
    assert np.array_equal(a.mem, b.mem)
    assert f[2] == f2 and f[3] == f3
    # and the put/get legs directly from the definition: PE1[300:364] = PE0[0:64]
    assert np.array_equal(a.pe(1)[300:364], init.reshape(npes, H)[0, 0:64])


def test_plain_script_race_free_invariants(orc):
    s = W.gen_plain_script(n_ops=3000)
    h = orc.Heap(s.npes, s.heap_bytes, s.heap)
    fetched = h.run_script(s.ops)
    ids = W.sync_interval_ids(s.ops)
    # per interval and word, fetch_adds fetch old values that form a chain: every
    # serial order of them is valid; checker confirms the script-order fetched values
    amo = np.isin(s.ops["kind"], W.AMO_KINDS)
    idx = np.nonzero(amo)[0]
    words = s.ops["pe"][idx].astype(np.int64) * s.heap_bytes + s.ops["dst"][idx].astype(np.int64)
    group = ids[idx] * (s.npes * s.heap_bytes) + words
    # starting value of each group = fetched value of its first op in script order
    w0 = np.zeros(len(idx), np.int64)
    firsts = {}
    for t, g in enumerate(group):
        firsts.setdefault(g, fetched[idx[t]])
        w0[t] = firsts[g]
    r = orc.check_serialisation(group, s.ops["kind"][idx], s.ops["operand"][idx],
                                s.ops["cond"][idx], fetched[idx], w0)
    assert r == 0
    # compare_swap outcomes occur both ways
    cs = idx[s.ops["kind"][idx] == W.OP_CSWAP]
    succ = fetched[cs] == s.ops["cond"][cs]
    assert succ.any() and (~succ).any()


# ----------------------------------------------------------------- halo-exchange stencil
def _jacobi_fixtures():
    grids, cur = [], None
    for line in open(os.path.join(GOLD, "jacobi_order.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "grid":
            cur = {"name": f[1], "g": np.zeros((int(f[2]), int(f[3])), np.float32), "expect": []}
            grids.append(cur)
        elif f[0] == "set":
            cur["g"][int(f[1]), int(f[2])] = np.float32(float.fromhex(f[3]))
        elif f[0] == "expect":
            cur["expect"].append((int(f[1]), int(f[2]), float.fromhex(f[3])))
    return grids


def test_halo_jacobi_operation_order_golden(orc):
    """The pairing (up + down) + (left + right), each add and the multiply rounded to
    binary32, against hand-derived values where other pairings round differently."""
    for fx in _jacobi_fixtures():
        out = orc.halo_jacobi(fx["g"], 1)
        for i, j, v in fx["expect"]:
            assert float(out[i, j]) == v, (fx["name"], i, j, float(out[i, j]), v)


def test_halo_jacobi_constant_delta_and_sum(orc):
    """A constant grid is a fixed point; a unit delta spreads 1/4 to exactly its four
    periodic neighbours (the corner wraps); the grid sum is conserved."""
    c = np.full((6, 10), 3.25, np.float32)
    assert np.array_equal(orc.halo_jacobi(c, 7), c)
    d = np.zeros((5, 7), np.float32)
    d[0, 0] = 1.0
    want = np.zeros_like(d)
    for i, j in ((1, 0), (4, 0), (0, 1), (0, 6)):
        want[i, j] = 0.25
    assert np.array_equal(orc.halo_jacobi(d, 1), want)
    x = W.normals_np(5, 12 * 9).astype(np.float32).reshape(12, 9)
    y = orc.halo_jacobi(x, 10)
    assert abs(float(y.astype(np.float64).sum()) - float(x.astype(np.float64).sum())) < 1e-4


def test_halo_jacobi_fourier_mode_decay(orc):
    """A separable Fourier mode cos(2 pi k x / Nx) cos(2 pi l y / Ny) is an eigenvector:
    each sweep scales it by (cos(2 pi k / Nx) + cos(2 pi l / Ny)) / 2."""
    ny, nx, k, l, T = 16, 24, 3, 2, 6
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    g0 = np.cos(2 * np.pi * k * xx / nx) * np.cos(2 * np.pi * l * yy / ny)
    lam = (np.cos(2 * np.pi * k / nx) + np.cos(2 * np.pi * l / ny)) / 2
    out = orc.halo_jacobi(g0.astype(np.float32), T).astype(np.float64)
    assert np.max(np.abs(out - lam ** T * g0)) < 2e-6


def test_amo_add_word_sums_matches_sequential_application(orc):
    """The per-word operand sums (vectorised) against the sequential C oracle: on an
    add-only stream over 2^10 words, init + sums is the final table for every word, with
    a first-op offset; on a mixed stream the sums count only the fetch_add ops, also on
    words that other kinds of op touch."""
    nlog, nw, oseed, tseed = 10, 1 << 10, 0x77, 0x99
    init = W.cb64_np(tseed, np.arange(nw, dtype=np.uint64)).view(np.int64)
    ops = W.amo_stream_np(8, 30000, nlog, only=W.AMO_CODE_FADD, offset=1000)
    t = init.copy()
    orc.amo_stream(t, ops, oseed, tseed, first_op=1000, want_fetched=False)
    words = np.arange(nw, dtype=np.int64)
    assert np.array_equal(init + orc.amo_add_word_sums(ops, 1000, oseed, words), t)
    sub = words[::7]
    assert np.array_equal(orc.amo_add_word_sums(ops, 1000, oseed, sub), (t - init)[::7])
    # mixed stream over 2^12 words (most words see several kinds): the sequential oracle
    # runs the same stream with every non-add op moved to a sentinel word (same position,
    # so the same draw), which leaves each other word at init + the sum of its fetch_adds
    nw = 1 << 12
    init = W.cb64_np(tseed, np.arange(nw, dtype=np.uint64)).view(np.int64)
    mixed = W.amo_stream_np(9, 30000, 12)
    code = mixed >> 27
    sentinel = np.uint32(nw - 1)
    moved = np.where(code == 0, mixed, (mixed & ~np.uint32((1 << 27) - 1)) | sentinel).astype(np.uint32)
    t = init.copy()
    orc.amo_stream(t, moved, oseed, tseed, want_fetched=False)
    w = (mixed & ((1 << 27) - 1)).astype(np.int64)
    checked = np.arange(nw - 1, dtype=np.int64)
    mixed_words = np.intersect1d(w[code == 0], w[code != 0])
    assert len(mixed_words) > 100          # words that see fetch_adds and other kinds
    s = orc.amo_add_word_sums(mixed, 0, oseed, checked)
    assert np.array_equal(init[checked] + s, t[checked])


# --------------------------------------------------------------------------- planted mistakes
# Each pin must catch a plausible mistake in the function it pins: the oracle function is
# replaced (on the CPU, in a stand-in module) by a variant with one such mistake, and at
# least one of its pins has to fail.
def _jacobi_with(mistake):
    def sweep(grid, iters):
        g = np.ascontiguousarray(grid, dtype=np.float32)
        q = np.float32(0.25)
        for _ in range(iters):
            up, dn = np.roll(g, 1, axis=0), np.roll(g, -1, axis=0)
            lf, rt = np.roll(g, 1, axis=1), np.roll(g, -1, axis=1)
            if mistake == "pairing":        # (up + left) + (down + right)
                g = q * ((up + lf) + (dn + rt))
            elif mistake == "weight":       # 1/5 instead of 1/4
                g = np.float32(0.2) * ((up + dn) + (lf + rt))
            elif mistake == "no_wrap":      # zero boundary instead of periodic
                up[0, :] = 0
                dn[-1, :] = 0
                lf[:, 0] = 0
                rt[:, -1] = 0
                g = q * ((up + dn) + (lf + rt))
            elif mistake == "axis":         # left/right taken along the rows' axis
                g = q * ((up + dn) + (np.roll(g, 1, axis=0) + rt))
            elif mistake == "fma":          # one rounding fewer (sum formed in binary64)
                g = (0.25 * ((up.astype(np.float64) + dn) + (lf.astype(np.float64) + rt))).astype(np.float32)
        return g
    return sweep


@pytest.mark.parametrize("mistake", ["pairing", "weight", "no_wrap", "axis", "fma"])
def test_halo_pins_catch_a_planted_mistake(mistake):
    import types

    fake = types.SimpleNamespace(halo_jacobi=_jacobi_with(mistake))
    caught = 0
    for pin in (test_halo_jacobi_operation_order_golden, test_halo_jacobi_constant_delta_and_sum,
                test_halo_jacobi_fourier_mode_decay):
        try:
            pin(fake)
        except AssertionError:
            caught += 1
    assert caught >= 1, mistake


def _word_sums_with(orc, mistake):
    def sums(ops, first_op, op_seed, words):
        w = (ops & np.uint32((1 << 27) - 1)).astype(np.int64)
        code = ops >> np.uint32(27)
        pos = np.searchsorted(words, w)
        pos[pos == len(words)] = 0
        hit = (words[pos] == w) & ((code == 0) if mistake != "all_codes" else True)
        i = np.nonzero(hit)[0]
        idx = i.astype(np.uint64) + (np.uint64(first_op) if mistake != "no_offset" else np.uint64(0))
        r = W.cb64_np(op_seed, idx)
        mask = np.uint64((1 << 20) - 1) if mistake != "mask" else np.uint64((1 << 21) - 1)
        v = (r & mask) + (np.uint64(1) if mistake != "no_plus_one" else np.uint64(0))
        return np.bincount(pos[i], weights=v.astype(np.float64), minlength=len(words)).astype(np.int64)
    return sums


@pytest.mark.parametrize("mistake", ["all_codes", "no_offset", "mask", "no_plus_one"])
def test_amo_sum_pin_catches_a_planted_mistake(orc, mistake):
    import types

    fake = types.SimpleNamespace(amo_stream=orc.amo_stream, amo_add_word_sums=_word_sums_with(orc, mistake))
    with pytest.raises(AssertionError):
        test_amo_add_word_sums_matches_sequential_application(fake)


# --------------------------------------------------------------------------- served results
def test_checksum32_closed_forms(orc):
    """Word i (little-endian) weighs 2i + 1, modulo 2^64: an empty buffer is 0; byte 3 of
    word 0 weighs 2^24; word 1 weighs 3 and word 2 weighs 5; n words of 2^32 - 1 give
    (2^32 - 1) * n^2 mod 2^64 (the first n odd numbers sum to n^2), which wraps for large n."""
    assert orc.checksum32(np.zeros(0, np.uint8)) == 0
    assert orc.checksum32(np.array([0, 0, 0, 1], np.uint8)) == 1 << 24
    assert orc.checksum32(np.array([7, 0, 0, 0, 1, 0, 0, 0, 2, 0, 0, 0], np.uint8)) == 7 + 3 * 1 + 5 * 2
    for n in (1, 2, 1000, 1 << 17):
        buf = np.full(4 * n, 0xFF, np.uint8)
        assert orc.checksum32(buf) == ((2 ** 32 - 1) * n * n) % 2 ** 64
    assert ((2 ** 32 - 1) * (1 << 17) ** 2) >= 2 ** 64   # the last case does wrap


def test_qsum_multi_member_golden(orc):
    """The hand-traced Neumaier rows of tests/golden/neumaier.txt that are exact in
    bfloat16, through the heap model's quantised all-reduce on a four-member team of
    stride 2 (PEs 1, 3, 5, 7 of 9): element k carries row k mod rows, member r holds the
    row's r-th value (rows of three get a trailing 0, which changes no sum) as a bf16 code
    times a power-of-two scale of its own per member and block (so the dequantised value
    is the traced one exactly), over two blocks with a ragged tail.  Every member's dst
    must equal the traced sum bitwise, and the PEs outside the team stay as they were.
    The order-sensitive rows fix the team-rank order, the distinct scales that each
    member's own scale is used."""
    rows = []
    for vals, want, _naive in _golden("neumaier.txt"):
        v = np.array([float(x) for x in vals.split(",")], np.float32)
        if np.all((v.view(np.uint32) & 0xFFFF) == 0):
            rows.append((np.concatenate([v, np.zeros(4 - len(v), np.float32)]), np.float32(float(want))))
    assert len(rows) >= 5
    npes, P, start, stride, n = 9, 4, 1, 2, 200
    H = 8192
    q_off, s_off, dst = 0, 1024, 2048
    rng = np.random.default_rng(17)
    init = rng.integers(0, 256, (npes, H), dtype=np.uint8)
    want = np.empty(n, np.float32)
    for r in range(P):
        p = start + r * stride
        scales = np.array([2.0 ** (3 * r - 4), 2.0 ** (5 - 2 * r)], np.float32)   # per block, distinct per member
        vals = np.array([rows[k % len(rows)][0][r] for k in range(n)], np.float32)
        codes = ((vals / np.repeat(scales, 128)[:n]).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
        assert np.array_equal(codes.astype(np.uint32) << 16, (vals / np.repeat(scales, 128)[:n]).view(np.uint32))
        init[p, q_off:q_off + 2 * n] = codes.view(np.uint8)
        init[p, s_off:s_off + 8] = scales.view(np.uint8)
    for k in range(n):
        want[k] = rows[k % len(rows)][1]
    h = orc.Heap(npes, H, init.reshape(-1).copy())
    h.qsum_reduce((start, stride, P), dst=dst, q_off=q_off, s_off=s_off, fmt=W.FMT_BF16, n=n)
    for p in range(npes):
        if p in range(start, start + P * stride, stride):
            assert np.array_equal(h.view(p, dst, n, np.float32).view(np.uint32), want.view(np.uint32)), p
            assert np.array_equal(h.pe(p)[:dst], init[p, :dst]) and np.array_equal(h.pe(p)[dst + 4 * n:], init[p, dst + 4 * n:])
        else:
            assert np.array_equal(h.pe(p), init[p]), p


def test_serve_request_results_by_kind(orc):
    """Each request kind's result from the operations it is defined by: put / get return
    the checksum of the source bytes (the copy is exact); alltoall the checksum of the
    team's blocks transposed (numpy); a reduction that of the heap model's team reduce; an
    AMO its fetched value, leaving the updated word."""
    lay = W.serve_layout(H=1 << 20, amo_words=64)
    npes = 6
    init = np.zeros((npes, lay.H), np.uint8)
    rng = np.random.default_rng(3)
    init[:, lay.ro_offset:lay.ro_offset + lay.ro_bytes] = rng.integers(0, 256, (npes, lay.ro_bytes), dtype=np.uint8)
    words = rng.integers(-2 ** 40, 2 ** 40, npes * lay.amo_words, dtype=np.int64)
    init[:, :8 * lay.amo_words] = words.view(np.uint8).reshape(npes, -1)
    src = lay.ro_offset + 4096

    def req(**kw):
        r = np.zeros((), W.REQ_DTYPE)
        for k, v in kw.items():
            r[k] = v
        return r

    # put from PE 4 to PE 1 and get by PE 2 from PE 5
    for kind, pe, iss, srcpe in ((1, 1, 4, 4), (2, 5, 2, 5)):
        h = orc.Heap(npes, lay.H, init.reshape(-1).copy())
        got = orc.serve_request(h, req(kind=kind, pe=pe, issuer=iss, n=1000, src=src), lay.amo_offset,
                                lay.amo_words, lay.arena_offset)
        assert got == orc.checksum32(init[srcpe, src:src + 1000])
    # alltoall over PEs 1..4, 64 bytes per pair
    P, m = 4, 64
    h = orc.Heap(npes, lay.H, init.reshape(-1).copy())
    got = orc.serve_request(h, req(kind=15, pe=1, issuer=P, n=m, src=src), lay.amo_offset, lay.amo_words,
                            lay.arena_offset)
    blocks = np.stack([init[1 + i, src:src + P * m].reshape(P, m) for i in range(P)])   # [i][j] = member i's block j
    want = np.concatenate([blocks[:, j, :].reshape(-1) for j in range(P)])               # member j gets blocks [i][j]
    assert got == orc.checksum32(want)
    # fp32 sum over PEs 0..2 of 256 elements
    P, n = 3, 256
    h = orc.Heap(npes, lay.H, init.reshape(-1).copy())
    got = orc.serve_request(h, req(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_F32, pe=0, issuer=P, n=n, src=src),
                            lay.amo_offset, lay.amo_words, lay.arena_offset)
    ref = orc.Heap(npes, lay.H, init.reshape(-1).copy())
    ref.reduce((0, 1, P), lay.arena_offset, src, n, W.DT_FLOAT, W.RED_SUM)
    assert got == orc.checksum32(ref.pe(0)[lay.arena_offset:lay.arena_offset + 4 * n])
    # bf16 payloads with per-128 scales over PEs 1..3, 256 elements (two blocks): codes of
    # small integers times power-of-two scales, so every partial sum is an exact binary32
    # integer and the Neumaier result is the plain integer sum; the scales sit at `cond`
    P, n = 3, 256
    ints = rng.integers(-200, 201, (P, n))
    scl = np.array([[2.0, 0.5], [4.0, 1.0], [0.25, 8.0]], np.float32)
    h = orc.Heap(npes, lay.H, init.reshape(-1).copy())
    sc_off = src + 4096
    for r in range(P):
        x = (ints[r] / np.repeat(scl[r], 128)).astype(np.float32)
        h.view(1 + r, src, n, np.uint16)[:] = (x.view(np.uint32) >> 16).astype(np.uint16)
        assert np.array_equal((x.view(np.uint32) & 0xFFFF), np.zeros(n, np.uint32))   # exact in bf16
        h.view(1 + r, sc_off, 2, np.float32)[:] = scl[r]
    got = orc.serve_request(h, req(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_BF16, pe=1, issuer=P, n=n, src=src,
                                   cond=sc_off), lay.amo_offset, lay.amo_words, lay.arena_offset)
    assert got == orc.checksum32(ints.sum(0).astype(np.float32).view(np.uint8))
    for r in range(P):
        assert np.array_equal(h.view(1 + r, lay.arena_offset, n, np.float32), ints.sum(0).astype(np.float32))
    # fetch_add on word 70 (PE 1, index 6): returns the old value, stores old + v
    h = orc.Heap(npes, lay.H, init.reshape(-1).copy())
    got = orc.serve_request(h, req(kind=5, dtype=W.DT_INT64, word=70, operand=12345), lay.amo_offset,
                            lay.amo_words, lay.arena_offset)
    assert got == int(words[70]) & (2 ** 64 - 1) or got == int(words[70])
    assert int(h.view(1, lay.amo_offset + 8 * 6, 1, np.int64)[0]) == int(words[70]) + 12345


def test_staged_requests_by_kind(orc):
    """Requests that stage their payload (flags bit 0): the region at the scratch offset is
    laid out as the request record defines it and the result follows from the payload
    words alone -- a put/get returns the checksum of the payload bytes, an alltoall that of
    the payload blocks transposed (numpy), a two-member fp32 reduction that of the
    elementwise binary32 sum of the two members' payload words (one RNE add), a two-member
    bf16 reduction that of the binary32 sum of the two dequantised values (Neumaier on two
    values is their correctly rounded sum), and a one-member reduction returns its own
    payload (fp32) -- with every PE outside the request untouched."""
    npes, H, R = 5, 1 << 16, 4096
    init = np.random.default_rng(21).integers(0, 256, (npes, H), dtype=np.uint8)

    def payload(seed, p, j0, count):
        return W.serve_payload_words(seed, p, j0, count)

    def req(**kw):
        r = np.zeros((), W.REQ_DTYPE)
        r["flags"] = 1
        r["word"] = 0x1234567
        for k, v in kw.items():
            r[k] = v
        return r

    def run(r):
        h = orc.Heap(npes, H, init.reshape(-1).copy())
        got = orc.serve_request(h, r, 0, 1, R, payload)
        return h, got

    def untouched(h, pes):
        for p in range(npes):
            if p not in pes:
                assert np.array_equal(h.pe(p), init[p]), p

    # put PE 3 -> PE 1 and get by PE 0 from PE 4, 1000 bytes: the payload of the source PE
    for kind, pe, iss, sp, dp in ((1, 1, 3, 3, 1), (2, 4, 0, 4, 0)):
        h, got = run(req(kind=kind, pe=pe, issuer=iss, n=1000))
        want = W.serve_payload_words(0x1234567, sp, 0, 250).view(np.uint8)
        assert got == orc.checksum32(want)
        assert np.array_equal(h.pe(dp)[R:R + 1000], want)                      # destination part
        assert np.array_equal(h.pe(sp)[R + 1008:R + 2008], want)              # source part at R + round16(n)
        untouched(h, (sp, dp))
    # alltoall over PEs 1..3, 48 bytes per pair: member j's block i = member i's payload block j
    P, m = 3, 48
    h, got = run(req(kind=15, pe=1, issuer=P, n=m))
    src = [W.serve_payload_words(0x1234567, 1 + i, 0, P * m // 4).view(np.uint8).reshape(P, m) for i in range(P)]
    want = np.concatenate([np.concatenate([src[i][j] for i in range(P)]) for j in range(P)])
    assert got == orc.checksum32(want)
    untouched(h, (1, 2, 3))
    # fp32 in place over PEs 2..3 (n = 300): one binary32 add per element
    n = 300
    h, got = run(req(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_F32, pe=2, issuer=2, n=n))
    x = [W.serve_payload_words(0x1234567, p, 0, n).view(np.float32) for p in (2, 3)]
    want = (x[0] + x[1]).astype(np.float32)
    assert got == orc.checksum32(want.view(np.uint8))
    assert np.array_equal(h.view(3, R, n, np.float32), want)
    # one member: its own payload
    h, got = run(req(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_F32, pe=4, issuer=1, n=n))
    assert got == orc.checksum32(W.serve_payload_words(0x1234567, 4, 0, n).view(np.uint8))
    # int64 in place over PEs 1..2, n = 50: word pairs as little-endian int64, summed with
    # two's-complement wraparound
    n = 50
    h, got = run(req(kind=16, dtype=W.DT_INT64, fmt=0, pe=1, issuer=2, n=n))
    x = [W.serve_payload_words(0x1234567, p, 0, 2 * n).view(np.int64) for p in (1, 2)]
    with np.errstate(over="ignore"):
        want = (x[0] + x[1]).astype(np.int64)
    assert got == orc.checksum32(want.view(np.uint8))
    assert np.array_equal(h.view(2, R, n, np.int64), want)
    # bf16 over PEs 0..1, n = 260 (three blocks): codes at R + 1040, scales at R + 1040 + 528
    n = 260
    h, got = run(req(kind=16, dtype=W.DT_FLOAT, fmt=W.FMT_BF16, pe=0, issuer=2, n=n))
    xs = []
    for p in (0, 1):
        w = W.serve_payload_words(0x1234567, p, 0, 528 // 4 + 3)
        codes = w[:n // 2].view(np.uint16)                                     # little-endian: low code first
        sc = w[528 // 4:528 // 4 + 3].view(np.float32)
        dec = (codes.astype(np.uint32) << np.uint32(16)).view(np.float32)
        xs.append((dec * np.repeat(sc, 128)[:n]).astype(np.float32))
    want = (xs[0] + xs[1]).astype(np.float32)
    assert got == orc.checksum32(want.view(np.uint8))
    assert np.array_equal(h.view(1, R, n, np.float32), want)
    untouched(h, (0, 1))


def _checksum_with(mistake):
    def cs(buf):
        b = np.ascontiguousarray(buf).tobytes()
        w = np.frombuffer(b, dtype=">u4" if mistake == "big_endian" else "<u4").astype(np.uint64)
        i = np.arange(len(w), dtype=np.uint64)
        k = np.uint64(2) * i + (np.uint64(0) if mistake == "even_weights" else np.uint64(1))
        if mistake == "no_wrap":
            return int(sum(int(a) * int(c) for a, c in zip(w, k)))
        with np.errstate(over="ignore"):
            return int(np.sum(w * k, dtype=np.uint64))
    return cs


@pytest.mark.parametrize("mistake", ["big_endian", "even_weights", "no_wrap"])
def test_checksum_pin_catches_a_planted_mistake(mistake):
    import types

    with pytest.raises(AssertionError):
        test_checksum32_closed_forms(types.SimpleNamespace(checksum32=_checksum_with(mistake)))


def test_binary64_references_are_exact_sums(orc):
    """The binary64 references behind the error gates: with few members and inputs whose
    products and partial sums are exact in binary64 (bf16 codes in [-1, 1] times a
    power-of-two scale; binary32 values with small integer numerators), the reference sum
    equals the exact rational sum and the magnitude sum the exact sum of magnitudes."""
    from fractions import Fraction as F

    P, n = 3, 256
    rng = np.random.default_rng(9)
    h = orc.Heap(P, 8192)
    # exponents 120..126 (magnitudes 2^-7 .. < 1), any mantissa and sign: three such values
    # times 1/4 sum exactly in binary64
    exps = rng.integers(120, 127, (P, n)).astype(np.uint16)
    codes = (exps << 7) | rng.integers(0, 128, (P, n)).astype(np.uint16) | (rng.integers(0, 2, (P, n)).astype(np.uint16) << 15)
    scale = np.float32(0.25)
    for r in range(P):
        h.view(r, 0, n, np.uint16)[:] = codes[r]
        h.view(r, 4096, 2, np.float32)[:] = scale
    y, a = h.qsum_ref64((0, 1, P), 0, 4096, W.FMT_BF16, n)
    for k in range(n):
        xs = [F(orc.bf16_decode(int(codes[r, k]))) * F(float(scale)) for r in range(P)]
        assert F(float(y[k])) == sum(xs) and F(float(a[k])) == sum(abs(x) for x in xs)
    vals = (rng.integers(-1000, 1000, (P, n)) / np.float32(64)).astype(np.float32)
    for r in range(P):
        h.view(r, 0, n, np.float32)[:] = vals[r]
    y, a = h.reduce_f32_ref64((0, 1, P), 0, n)
    for k in range(n):
        xs = [F(float(vals[r, k])) for r in range(P)]
        assert F(float(y[k])) == sum(xs) and F(float(a[k])) == sum(abs(x) for x in xs)
