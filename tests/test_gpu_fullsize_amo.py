"""Full-size parity of the AMO stress stream in the launch configuration the benchmark
times: 1024 PEs (one CTA each, or the block-combined persistent grid) over a 2^27-word
int64 table, 2^30 ops.  The oracle checks sampled words:
  * a fetch_add-only Zipf(1.1) stream, block-combined: every sampled word -- 2^16 drawn
    at random plus the 64 hottest, which take about two fifths of all ops -- ends at its
    initial value plus the sum of the operands aimed at it;
  * the mixed streams (uniform and Zipf; plain and block-combined): all ops on 2^16
    sampled words admit one serial order, given their fetched values and the words'
    final values (the oracle's serialisation checker).
The streams are drawn on the host by a spawned process pool, in chunks, as the benchmark
draws them."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

NOPS = 1 << 30
NPES, WPP = 1024, 1 << 17
NWORDS = NPES * WPP
CHUNK = 1 << 24
SAMPLE = 1 << 16
MAX_GROUP = 1 << 14   # sampled words with more ops than this are left to the add-only check


def _chunk_ops(seed, dist, only, off, count):
    return W.amo_stream_np(seed, count, 27, dist=dist, offset=off, only=only)


def _chunk_sums(seed, dist, only, off, count, op_seed, words):
    import oracle

    return oracle.amo_add_word_sums(_chunk_ops(seed, dist, only, off, count), off, op_seed, words)


def _chunk_hits(seed, dist, off, count, words):
    """(op index, word, code) of the chunk's ops that target one of ``words``."""
    ops = _chunk_ops(seed, dist, None, off, count)
    w = (ops & np.uint32(NWORDS - 1)).astype(np.int64)
    pos = np.searchsorted(words, w)
    pos[pos == len(words)] = 0
    i = np.nonzero(words[pos] == w)[0]
    return i.astype(np.int64) + off, w[i], (ops[i] >> np.uint32(27)).astype(np.int64)


@pytest.fixture(scope="module")
def pool():
    p = cf.ProcessPoolExecutor(max(1, min(16, os.cpu_count() or 1)), mp_context=mp.get_context("spawn"))
    yield p
    p.shutdown()


@pytest.fixture(scope="module")
def table(sg):
    torch.cuda.set_device(0)
    heap = sg.Heap(NPES, WPP * 8 + 16384)
    tseed = W.derive_seed("amo-table")
    parts = heap.partitions()

    def reset():
        for p0 in range(0, NPES, 128):
            idx = torch.arange(p0 * WPP, (p0 + 128) * WPP, dtype=torch.int64, device="cuda")
            parts[p0:p0 + 128, :WPP * 8].view(torch.int64).copy_(W.cb64_torch(tseed, idx).view(128, WPP))
        torch.cuda.synchronize()

    yield heap, tseed, reset
    heap.close()


def _stream(pool, seed, dist, only=None):
    out = np.empty(NOPS, np.uint32)
    futs = {pool.submit(_chunk_ops, seed, dist, only, c, CHUNK): c for c in range(0, NOPS, CHUNK)}
    for f, c in futs.items():
        out[c:c + CHUNK] = f.result()
    return torch.from_numpy(out.view(np.int32)).cuda()


def _words_at(heap, words):
    flat = heap.partitions()[:, :WPP * 8].view(torch.int64).reshape(-1)
    return flat[torch.from_numpy(words).cuda()].cpu().numpy()


def _random_words(tag):
    w = W.cb64_np(W.derive_seed(tag), np.arange(SAMPLE, dtype=np.uint64)) & np.uint64(NWORDS - 1)
    return np.unique(w.astype(np.int64))


def _hottest_zipf_words(k):
    r = np.arange(k, dtype=np.uint64)   # ranks 1..k, minus one
    return np.unique((((r * np.uint64(W.ZIPF_MULT)) & np.uint64(NWORDS - 1)) ^ np.uint64(W.ZIPF_XOR & (NWORDS - 1))).astype(np.int64))


def test_fetch_add_zipf_block_combined_sums(sg, orc, pool, table):
    heap, tseed, reset = table
    reset()
    seed, oseed = W.derive_seed("amo-zipf-add"), W.derive_seed("amo-ops")
    dops = _stream(pool, seed, "zipf", only=W.AMO_CODE_FADD)
    words = np.union1d(_random_words("amo-sample-add"), _hottest_zipf_words(64))
    init = _words_at(heap, words)
    sg.clear_status()
    sg.amo_stream(heap.base, WPP, dops, NOPS, oseed, tseed, None, flags=sg.AMO_COMBINE_BLOCK)
    torch.cuda.synchronize()
    assert sg.get_status()[0] == 0
    del dops
    got = _words_at(heap, words)
    sums = np.zeros(len(words), np.int64)
    futs = [pool.submit(_chunk_sums, seed, "zipf", W.AMO_CODE_FADD, c, CHUNK, oseed, words) for c in range(0, NOPS, CHUNK)]
    for f in futs:
        sums += f.result()
    assert sums.sum() > NOPS // 8   # the hot words carry a large share of the stream
    assert np.array_equal(got, init + sums)


@pytest.mark.parametrize("dist,flag_list", [("zipf", (0, 2)), ("uniform", (2,))])
def test_mixed_stream_serialisable_on_sampled_words(sg, orc, pool, table, dist, flag_list):
    heap, tseed, reset = table
    seed, oseed = W.derive_seed("amo-" + dist), W.derive_seed("amo-ops")
    dops = _stream(pool, seed, dist)
    words = _random_words("amo-sample-" + dist)
    hits = [pool.submit(_chunk_hits, seed, dist, c, CHUNK, words) for c in range(0, NOPS, CHUNK)]
    parts = [f.result() for f in hits]
    idx = np.concatenate([p[0] for p in parts])
    w = np.concatenate([p[1] for p in parts])
    code = np.concatenate([p[2] for p in parts])
    # leave out the few sampled words whose groups are too large for the exhaustive check
    uw, cnt = np.unique(w, return_counts=True)
    keep = np.isin(w, uw[cnt <= MAX_GROUP])
    idx, w, code = idx[keep], w[keep], code[keep]
    assert len(idx) > 10000
    checked = np.unique(w)
    init_all = W.cb64_np(tseed, checked.astype(np.uint64)).view(np.int64)
    init = init_all[np.searchsorted(checked, w)]
    r = W.cb64_np(oseed, idx.astype(np.uint64))
    operand = np.where(code == 0, (r % np.uint64(1 << 20)) + np.uint64(1), np.where(r == 0, np.uint64(1), r)).view(np.int64)
    kind = np.array([W.OP_FADD, W.OP_CSWAP, W.OP_FXOR])[code]
    fetched = torch.empty(NOPS, dtype=torch.int64, device="cuda")
    for flags in flag_list:
        reset()
        sg.clear_status()
        sg.amo_stream(heap.base, WPP, dops, NOPS, oseed, tseed, fetched, flags=flags)
        torch.cuda.synchronize()
        assert sg.get_status()[0] == 0
        f = fetched[torch.from_numpy(idx).cuda()].cpu().numpy()
        final = _words_at(heap, checked)[np.searchsorted(checked, w)]
        assert orc.check_serialisation(w, kind, operand, init, f, init, final) == 0, flags
    del dops, fetched
