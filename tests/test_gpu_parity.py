"""Parity of the CUDA path with the CPU oracle, byte for byte.

Every result of the path is an exact permutation of bytes with a unique
answer, so the tolerance is zero: counts, offsets and the sorted stream must
equal the oracle's exactly.  Inputs are seeded: the paper-sized synthetic
documents, and adversarial cases for each kernel (chunk and tile boundaries,
ragged tails, every word length 1..255, key widths 1..32 u64 words, giant
single buckets, all-equal keys, unaligned device pointers, empty inputs).
"""
import random

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def assert_same(got, exp, label=""):
    assert got.n_words == exp["n_words"], label
    assert got.max_len == exp["max_len"], label
    assert got.stream_bytes == exp["stream_bytes"], label
    assert np.array_equal(got.counts, exp["counts"]), label
    assert np.array_equal(got.offsets, exp["offsets"]), label
    assert np.array_equal(got.stream, exp["stream"]), label


def assert_same_dev(dev, exp, label=""):
    assert dev["n_words"] == exp["n_words"] and dev["max_len"] == exp["max_len"], label
    assert np.array_equal(dev["counts"].cpu().numpy().astype(np.uint64), exp["counts"]), label
    assert np.array_equal(dev["offsets"].cpu().numpy().astype(np.uint32), exp["offsets"]), label
    assert np.array_equal(dev["stream"].cpu().numpy(), exp["stream"]), label


@pytest.fixture(scope="module", params=["dedupe=2", "dedupe=0"])
def ctx(bsort_gpu, request):
    """A context with the duplicate-aware sort of the large buckets (the
    default) and one with merge passes instead: every test runs on both."""
    c = bsort_gpu.Context(tune_table=request.param)
    yield c
    c.close()


HAND = [
    b"Hello, world! The cat-sat\non a mat; The end.",
    b"", b"!!! ... ---", b" \t\n\x0b\x0c\r ", b"a\tb\r\nc", b"\xc3\xa9t\xc3\xa9", b"don't can't",
    b"abc123 456", b"a\x00b", b"Zebra apple", b"b a b a", b"zz y xxx", b"q", b"x" * 255,
]


@pytest.mark.parametrize("i", range(len(HAND)))
def test_hand_cases(ctx, oracle_mod, i):
    data = HAND[i]
    assert_same(ctx.text(data), oracle_mod.bubble(data), repr(data))


def test_hand_example_values(ctx):
    r = ctx.text(b"Hello, world! The cat-sat\non a mat; The end.")
    assert r.counts.tolist() == [0, 1, 1, 4, 0, 2, 1]
    assert r.stream.tobytes() == b"aonTheTheendmatHelloworldcatsat"
    assert r.offsets.tolist() == [0, 1, 3, 6, 9, 12, 15, 20, 25, 31]


@pytest.mark.parametrize("name", ["plain_190k", "plain_1m38"])
def test_paper_sized_documents(ctx, oracle_mod, synth_mod, name):
    import torch

    data = synth_mod.plain(name)
    exp = oracle_mod.stable(data, nthreads=8)
    assert_same(ctx.text(data), exp, name)
    assert_same_dev(ctx.text_device(torch.from_numpy(data).cuda()), exp, name)
    torch.cuda.synchronize()
    if name == "plain_190k":
        assert_same(ctx.text(data), oracle_mod.bubble(data, nthreads=8), name + " vs bubble")


def test_repeat_calls_identical(ctx, synth_mod):
    data = synth_mod.plain("plain_190k")
    a = ctx.text(data)
    b = ctx.text(data)
    assert np.array_equal(a.stream, b.stream) and np.array_equal(a.offsets, b.offsets)


def _fuzz_bytes(rng: random.Random, n: int) -> bytes:
    pool = (b"abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ" * 4 + b" \t\n\x0b\x0c\r" * 3
            + b".,;:?!\"'-0123456789" + bytes(range(128, 256, 5)) + b"\x00\x7f")
    return bytes(rng.choice(pool) for _ in range(n))


@pytest.mark.parametrize("seed", range(12))
def test_fuzz_random_bytes(ctx, oracle_mod, seed):
    rng = random.Random(seed)
    data = _fuzz_bytes(rng, rng.choice([1, 15, 16, 17, 1000, 16383, 16384, 16385, 50_000, 200_000]))
    assert_same(ctx.text(data), oracle_mod.stable(data), f"seed {seed}")


def test_every_length_and_key_width(ctx, oracle_mod):
    # words of every length 1..255: all six key widths (1, 2, 4, 8, 16, 32 u64)
    # and the 8/9, 16/17, 32/33, 64/65, 128/129 boundaries
    rng = random.Random(3)
    words = []
    for L in range(1, 256):
        for _ in range(rng.randint(1, 40)):
            words.append(bytes(rng.choice(b"abcXYZ") for _ in range(L)))
    rng.shuffle(words)
    data = b" ".join(words)
    assert_same(ctx.text(data), oracle_mod.stable(data, nthreads=8))


def test_long_words_share_prefixes(ctx, oracle_mod):
    # multi-word keys that agree on the first words and differ late
    rng = random.Random(4)
    words = []
    for L in (9, 16, 17, 24, 31, 32, 33, 40, 64, 65, 100, 128, 129, 200, 255):
        stem = bytes(rng.choice(b"ab") for _ in range(L - 1))
        for _ in range(300):
            words.append(stem + bytes([rng.choice(b"abAB")]))
            words.append(bytes(rng.choice(b"ab") for _ in range(L)))
    rng.shuffle(words)
    data = b"\n".join(words)
    assert_same(ctx.text(data), oracle_mod.stable(data, nthreads=8))


def test_giant_single_bucket(ctx, oracle_mod):
    # 600k five-letter words: one bucket spanning ~300 tiles and 9 merge passes
    rng = np.random.default_rng(5)
    letters = rng.integers(97, 123, size=(600_000, 5), dtype=np.uint8)
    data = np.concatenate([letters, np.full((600_000, 1), 32, np.uint8)], axis=1).reshape(-1)
    assert_same(ctx.text(data), oracle_mod.stable(data, nthreads=8))


def test_pipelined_merge_passes(ctx, oracle_mod):
    """Enough one-word keys for the pipelined merge (cut kernel, then merge
    kernel with two buffers): one bucket of 3M words (about 1,500 tiles), one
    that finishes after two passes and sits idle in the later ones, and one of
    an odd number of runs (a run carried through a pass alone)."""
    rng = np.random.default_rng(9)
    parts = []
    for L, n in ((5, 3_000_000), (3, 40_000), (7, 17 * 2048 * 8 + 5)):
        letters = rng.choice(np.frombuffer(b"abcdefgh", np.uint8), size=(n, L))
        parts.append(np.concatenate([letters, np.full((n, 1), 32, np.uint8)], axis=1).reshape(-1))
    cut = 6 * 1_000_000  # whole words of the first part
    data = np.concatenate([parts[1], parts[0][:cut], parts[2], parts[0][cut:]])
    assert_same(ctx.text(data), oracle_mod.stable(data, nthreads=8))


def test_all_equal_keys_and_reverse_order(ctx, oracle_mod):
    data = b" ".join([b"same"] * 100_000 + [b"%04d" % 0 + b"z"] + [bytes([122 - i % 26]) * 3 for i in range(50_000)])
    assert_same(ctx.text(data), oracle_mod.stable(data))


def test_words_straddling_chunks(ctx, oracle_mod):
    # punctuation runs inside words that cross 16 KiB chunk boundaries
    parts = [b"a" + b"-" * 40_000 + b"b", b"  ", b"xy" + b"." * 16_383 + b"z", b" ", b"q" * 200 + b"'" * 5 + b"r" * 55]
    data = b"\n".join([b"".join(parts)] * 3)
    exp = oracle_mod.stable(data)
    assert exp["max_len"] == 255
    assert_same(ctx.text(data), exp)
    assert oracle_mod.tokenize(data)[0] == b"ab"


@pytest.mark.parametrize("offset", [0, 1, 3, 7, 8, 13, 15])
def test_unaligned_device_input(ctx, oracle_mod, synth_mod, offset):
    import torch

    data = synth_mod.text(synth_mod.TAG_FUZZ, 100 + offset, 70_001 + offset, 900, 3.7, 20)
    buf = torch.zeros(data.size + 64, dtype=torch.uint8, device="cuda")
    buf[offset:offset + data.size] = torch.from_numpy(data).cuda()
    buf[:offset] = ord("z")  # bytes before and after the document must not leak in
    buf[offset + data.size:] = ord("z")
    dev = ctx.text_device(buf[offset:offset + data.size])
    torch.cuda.synchronize()
    assert_same_dev(dev, oracle_mod.stable(data), f"offset {offset}")


def test_empty_device_input(ctx):
    import torch

    dev = ctx.text_device(torch.zeros(0, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    assert dev["n_words"] == 0 and dev["max_len"] == 0
    assert dev["counts"].cpu().tolist() == [0] and dev["offsets"].cpu().tolist() == [0]


def test_word_too_long(bsort_gpu):
    with bsort_gpu.Context(l_cap=10) as c:
        assert c.text(b"abcdefghij ok").n_words == 2
        with pytest.raises(bsort_gpu.BsortError) as e:
            c.text(b"ok abcdefghijk ok")
        assert e.value.status == bsort_gpu.BSORT_E_WORD_TOO_LONG
        # the context stays usable
        assert c.text(b"b a").stream.tobytes() == b"ab"
    with bsort_gpu.Context() as c:
        with pytest.raises(bsort_gpu.BsortError) as e:
            c.text(b"x" * 256)
        assert e.value.status == bsort_gpu.BSORT_E_WORD_TOO_LONG


def test_no_offsets_mode(bsort_gpu, oracle_mod, synth_mod):
    data = synth_mod.plain("plain_190k")
    with bsort_gpu.Context(want_offsets=False) as c:
        r = c.text(data)
    exp = oracle_mod.stable(data)
    assert r.offsets is None
    assert np.array_equal(r.stream, exp["stream"]) and np.array_equal(r.counts, exp["counts"])


def test_batch_equals_single(ctx, oracle_mod, synth_mod):
    rng = random.Random(9)
    docs = [synth_mod.batch_doc(*s) for s in synth_mod.batch_shapes(40)]
    docs[3] = np.zeros(0, np.uint8)
    docs[7] = np.frombuffer(b"  ..  ", np.uint8)
    docs[11] = np.frombuffer(_fuzz_bytes(rng, 5000), np.uint8)
    docs[12] = np.frombuffer(b"word", np.uint8)
    st, rs = ctx.batch(docs)
    assert st == 0, ctx.last_error()
    for i, d in enumerate(docs):
        exp = oracle_mod.stable(d, nthreads=8)
        assert_same(rs[i], exp, f"doc {i}")
        assert_same(ctx.text(d), exp, f"doc {i} alone")


def test_batch_meta_region_copied(ctx, oracle_mod, synth_mod):
    """96 documents: a meta region (totals, bases, histograms) over 64 KB,
    which reaches the host by a copy rather than from K1's last CTA (the
    batches above are small enough for the direct path)."""
    docs = [synth_mod.batch_doc(*s) for s in synth_mod.batch_shapes(96)]
    st, rs = ctx.batch(docs)
    assert st == 0, ctx.last_error()
    for i, d in enumerate(docs):
        assert_same(rs[i], oracle_mod.stable(d, nthreads=8), f"doc {i}")


def test_page_locked_and_packed_host_inputs(ctx, bsort_gpu, oracle_mod, synth_mod):
    """Host inputs read in place from page-locked memory, packed documents
    moved as one region (page-locked or not), and scattered ones gathered:
    every form gives the oracle's result."""
    doc = synth_mod.plain("plain_190k")
    pinned = bsort_gpu.pinned_empty(doc.size)
    pinned[:] = doc
    exp = oracle_mod.stable(doc, nthreads=8)
    assert_same(ctx.text(pinned), exp)
    assert_same(ctx.text(pinned, copy=False), exp)
    docs = [synth_mod.batch_doc(*s) for s in synth_mod.batch_shapes(12)]
    docs.insert(3, np.zeros(0, np.uint8))
    docs.insert(7, np.frombuffer(b"!! ??", np.uint8))
    exps = [oracle_mod.stable(d, nthreads=8) for d in docs]
    for form in (bsort_gpu.pack_host(docs), bsort_gpu.pack_host(docs, pinned=False), docs):
        st, rs = ctx.batch(form)
        assert st == 0
        for i, (r, e) in enumerate(zip(rs, exps)):
            assert_same(r, e, f"doc {i}")


def test_batch_reports_failing_document(bsort_gpu, oracle_mod):
    docs = [b"fine words here", b"x" * 30, b"also fine"]
    with bsort_gpu.Context(l_cap=20) as c:
        st, rs = c.batch(docs)
    assert st == bsort_gpu.BSORT_E_WORD_TOO_LONG
    assert [r.status for r in rs] == [0, bsort_gpu.BSORT_E_WORD_TOO_LONG, 0]
    assert_same(rs[0], oracle_mod.stable(docs[0]))
    assert_same(rs[2], oracle_mod.stable(docs[2]))


@pytest.mark.slow
def test_plain_256m_full(ctx, oracle_mod, synth_mod):
    """The 256 MiB workload through the device entry point, as the benchmark
    runs it, against the oracle's stable_sort path on every byte."""
    import torch

    data = synth_mod.plain("plain_256m")
    dev = ctx.text_device(torch.from_numpy(data).cuda())
    torch.cuda.synchronize()
    exp = oracle_mod.stable(data, nthreads=oracle_mod.max_threads())
    assert_same_dev(dev, exp, "plain_256m")
    assert exp["max_len"] > 16  # multi-word keys are exercised


def test_batch_device_packed_unaligned(ctx, oracle_mod, synth_mod):
    """Documents packed back to back in one device buffer (so most start at
    unaligned addresses), with empty and punctuation-only documents among
    them; each result equals the oracle's for that document alone."""
    import torch

    docs = [synth_mod.batch_doc(*s) for s in synth_mod.batch_shapes(24)]
    docs.insert(5, np.zeros(0, np.uint8))
    docs.insert(9, np.frombuffer(b"!!", np.uint8))
    docs.append(np.frombuffer(b"tail", np.uint8))
    lens = [d.size for d in docs]
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.uint64).tolist()
    base = torch.from_numpy(np.concatenate(docs)).cuda()
    st, outs = ctx.batch_device(base, offs, lens)
    torch.cuda.synchronize()
    assert st == 0, ctx.last_error()
    for i, d in enumerate(docs):
        assert_same_dev(outs[i], oracle_mod.stable(d, nthreads=8), f"doc {i}")


def test_batch_device_reports_failing_document(bsort_gpu, oracle_mod):
    import torch

    docs = [b"alpha beta", b"x" * 40, b"", b"gamma"]
    lens = [len(d) for d in docs]
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.uint64).tolist()
    base = torch.frombuffer(bytearray(b"".join(docs)), dtype=torch.uint8).cuda()
    with bsort_gpu.Context(l_cap=30) as c:
        st, outs = c.batch_device(base, offs, lens)
        torch.cuda.synchronize()
    assert st == bsort_gpu.BSORT_E_WORD_TOO_LONG
    assert [o["status"] for o in outs] == [0, bsort_gpu.BSORT_E_WORD_TOO_LONG, 0, 0]
    for i in (0, 2, 3):
        assert_same_dev(outs[i], oracle_mod.stable(docs[i]), f"doc {i}")


@pytest.mark.parametrize("W,lengths", [(1, (3, 4, 5, 6, 7, 8)), (2, (9, 10, 12, 13, 15, 16)),
                                       (4, (17, 20, 24, 28, 31, 32))])
def test_bucket_sizes_at_kernel_thresholds(ctx, oracle_mod, W, lengths):
    """Buckets whose sizes sit at and around every K4 boundary for their key
    width: the warp sort (32 lanes x 8/W keys), one CTA tile (2048/W keys),
    clusters of 2, 4 and 8 tiles, and the first merge pass."""
    rng = np.random.default_rng(100 + W)
    warp, tile = 32 * (8 // W), 2048 // W
    sizes = [1, warp - 1, warp, warp + 1, tile, tile + 1, 2 * tile + 1, 4 * tile + 1, 8 * tile, 8 * tile + 1,
             17 * tile + 5]
    words = []
    for j, n in enumerate(sizes):
        L = lengths[j % len(lengths)] if j < len(lengths) else lengths[j % len(lengths)]
        # a small alphabet gives duplicates and long shared prefixes
        letters = rng.choice(np.frombuffer(b"abAB", np.uint8), size=(n, L))
        words.extend(bytes(r) for r in letters)
    order = rng.permutation(len(words))
    data = b" ".join(words[i] for i in order)
    assert_same(ctx.text(data), oracle_mod.stable(data, nthreads=8))


def test_serving_results_equal_alone(bsort_gpu, oracle_mod, synth_mod):
    """Continuous batching: requests submitted from one thread while another
    polls; every result (including a failing one and an empty one) equals the
    oracle's for that document alone, whatever batch it was served in."""
    import threading
    import time

    docs = [synth_mod.batch_doc(*s) for s in synth_mod.batch_shapes(30)]
    docs[4] = np.zeros(0, np.uint8)
    docs[7] = np.frombuffer(b"fine " + b"y" * 300 + b" words", np.uint8)  # 300 letters: too long
    results, lat = {}, {}
    with bsort_gpu.Context() as c:
        c.serve_start(hbm_budget=1 << 30, workers=2, max_batch_docs=8)

        def producer():
            rng = random.Random(1)
            for i, d in enumerate(docs):
                assert c.submit(d, i) == 0
                time.sleep(rng.random() * 0.003)

        th = threading.Thread(target=producer)
        th.start()
        deadline = time.time() + 120
        while len(results) < len(docs) and time.time() < deadline:
            for tag, res, ns in c.poll(16):
                results[tag] = res
                lat[tag] = ns
            time.sleep(0.001)
        th.join()
        c.serve_stop()
    assert sorted(results) == list(range(len(docs)))
    for i, d in enumerate(docs):
        if i == 7:
            assert results[i].status == bsort_gpu.BSORT_E_WORD_TOO_LONG
            continue
        assert results[i].status == 0
        assert_same(results[i], oracle_mod.stable(d, nthreads=8), f"request {i}")
        assert lat[i] > 0


def test_serving_views_held_until_released(bsort_gpu, oracle_mod, synth_mod):
    """Results polled as views of the server's buffers (no copy) stay intact
    across later polls and batches until released, also when released out of
    order from other threads; released buffers go back to the workers, whose
    later batches write into them; results still held survive serve_stop."""
    import threading
    import time

    docs = [synth_mod.batch_doc(*s) for s in synth_mod.batch_shapes(48)]
    with bsort_gpu.Context() as c:
        c.serve_start(hbm_budget=1 << 30, workers=2, max_batch_docs=4)
        for i, d in enumerate(docs):
            assert c.submit(d, i) == 0
        held = {}
        deadline = time.time() + 120
        while len(held) < len(docs) and time.time() < deadline:
            for tag, res, _ in c.poll(5, copy=False):
                held[tag] = res
            time.sleep(0.001)
        assert sorted(held) == list(range(len(docs)))
        # every view still matches after all the polls; release half of them
        # from two threads, in scrambled order
        for i, d in enumerate(docs):
            assert_same(held[i], oracle_mod.stable(d, nthreads=8), f"held request {i}")
        first = [t for t in range(len(docs)) if t % 2 == 0]
        random.Random(5).shuffle(first)
        ths = [threading.Thread(target=lambda ts: [c.release(held.pop(t)) for t in ts], args=(first[k::2],))
               for k in range(2)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        # more batches now reuse the released buffers; the views still held
        # must not change
        for i, d in enumerate(docs):
            assert c.submit(d, 1000 + i) == 0
        again = {}
        deadline = time.time() + 120
        while len(again) < len(docs) and time.time() < deadline:
            for tag, res, _ in c.poll(8):  # copied out and released at once
                again[tag] = res
            time.sleep(0.001)
        c.serve_stop()
        for i, d in enumerate(docs):
            exp = oracle_mod.stable(d, nthreads=8)
            assert_same(again[1000 + i], exp, f"second round {i}")
            if i in held:
                assert_same(held[i], exp, f"still held {i}")
        for t in list(held):
            c.release(held.pop(t))


def test_serving_borrowed_inputs(bsort_gpu, oracle_mod, synth_mod):
    """Requests submitted without a copy: page-locked documents (read in place
    by the copy engine, back to back or scattered by the submission order) and
    pageable ones, mixed with copied submissions; every result equals the
    oracle's, and the context drops its references once the results are
    polled."""
    import time

    docs = [synth_mod.batch_doc(*s) for s in synth_mod.batch_shapes(36)]
    docs[5] = np.zeros(0, np.uint8)
    pinned = bsort_gpu.pack_host(docs)
    order = list(range(len(docs)))
    random.Random(9).shuffle(order)
    with bsort_gpu.Context() as c:
        c.serve_start(hbm_budget=1 << 30, workers=2, max_batch_docs=6)
        for k, i in enumerate(order):
            mode = k % 3
            if mode == 0:
                assert c.submit(pinned[i], i, borrow=True) == 0
            elif mode == 1:
                assert c.submit(np.array(docs[i]), i, borrow=True) == 0
            else:
                assert c.submit(docs[i], i) == 0
        got = {}
        deadline = time.time() + 120
        while len(got) < len(docs) and time.time() < deadline:
            for tag, res, _ in c.poll(7):
                got[tag] = res
            time.sleep(0.001)
        c.serve_stop()
        assert not c._borrowed
    assert sorted(got) == list(range(len(docs)))
    for i, d in enumerate(docs):
        assert got[i].status == 0
        assert_same(got[i], oracle_mod.stable(d, nthreads=8), f"request {i}")


def test_serving_rejects_over_budget(bsort_gpu):
    with bsort_gpu.Context() as c:
        c.serve_start(hbm_budget=1 << 20, workers=1)
        assert c.submit(np.zeros(1 << 20, np.uint8), 1) == bsort_gpu.BSORT_E_TOO_LARGE
        assert c.submit(b"small doc", 2) == 0
        c.serve_stop()
        got = c.poll(8)
        assert [t for t, _, _ in got] == [2] and got[0][1].words() == [b"doc", b"small"]


def _device_span(bs, torch, ptrs_and_sizes, itemsize, typestr):
    """Host copy of one device buffer spanning [first pointer, last pointer +
    its size): the outputs of a batch lie in one buffer per kind, in order."""
    lo = min(p for p, n in ptrs_and_sizes if n)
    hi = max(p + n * itemsize for p, n in ptrs_and_sizes if n)
    t = torch.as_tensor(bs._DevView(lo, (hi - lo) // itemsize, typestr), device="cuda")
    return lo, t.cpu().numpy()


@pytest.mark.slow
def test_batch_4096_full(bsort_gpu, oracle_mod, synth_mod):
    """All 4,096 documents of the batch workload (2.07 GB) in one
    bsort_batch_device call, as the benchmark runs it; every document's
    counts, offsets and stream byte for byte against the oracle's result for
    that document alone."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    import torch

    cores = os.cpu_count() or 8
    docs = synth_mod.batch(None, threads=cores)
    assert len(docs) == 4096
    lens = [int(d.size) for d in docs]
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.uint64).tolist()
    base = torch.from_numpy(np.concatenate(docs)).cuda()
    with bsort_gpu.Context() as c:
        st, rs = c.batch_device_raw(base, offs, lens)
        torch.cuda.synchronize()
        assert st == 0, c.last_error()
        assert all(r.status == 0 for r in rs)
        # (signed views on the device: torch copies int64/int32 everywhere)
        c0, counts = _device_span(bsort_gpu, torch, [(r.counts, r.max_len + 1) for r in rs], 8, "<i8")
        o0, offsets = _device_span(bsort_gpu, torch, [(r.offsets, r.n_words + 1) for r in rs], 4, "<i4")
        counts, offsets = counts.view(np.uint64), offsets.view(np.uint32)
        s0, stream = _device_span(bsort_gpu, torch, [(r.stream, r.stream_bytes) for r in rs], 1, "|u1")
    del base

    def check(i):
        r, exp = rs[i], oracle_mod.stable(docs[i])
        if (r.n_words, r.max_len, r.stream_bytes) != (exp["n_words"], exp["max_len"], exp["stream_bytes"]):
            return i
        a = (r.counts - c0) // 8
        b = (r.offsets - o0) // 4
        s = r.stream - s0 if r.stream_bytes else 0
        same = (np.array_equal(counts[a:a + r.max_len + 1], exp["counts"])
                and np.array_equal(offsets[b:b + r.n_words + 1], exp["offsets"])
                and np.array_equal(stream[s:s + r.stream_bytes], exp["stream"]))
        return None if same else i

    with ThreadPoolExecutor(cores) as ex:
        bad = [i for i in ex.map(check, range(len(docs))) if i is not None]
    assert bad == [], f"documents differing from the oracle: {bad[:20]}"


@pytest.mark.parametrize("case", ["one_word", "two_words", "hot_and_cold", "all_distinct_wide", "hot_and_cold_wide"])
def test_duplicate_aware_extremes(ctx, oracle_mod, case):
    """Large buckets at the extremes of repetition: one word repeated 3M
    times (one distinct key whose count spans every tile), two words, a few
    hot words among many cold ones, distinct words of 33..64 letters (keys of
    8 words, whose distinct-key entries take the 16-word sort), and hot and
    cold words of 12 and 24 letters (keys of 2 and 4 words, whose table
    slots publish their key after a claim, so that readers of a hot word wait
    for it)."""
    rng = np.random.default_rng({"one_word": 1, "two_words": 2, "hot_and_cold": 3, "all_distinct_wide": 4,
                                 "hot_and_cold_wide": 5}[case])
    if case == "one_word":
        data = b"hello " * 3_000_000
    elif case == "two_words":
        words = np.where(rng.random(2_000_000) < 0.3, 1, 0)
        data = b" ".join([b"Alpha", b"alpha"][i] for i in words)
    elif case == "hot_and_cold":
        cold = rng.choice(np.frombuffer(b"abcdefghij", np.uint8), size=(400_000, 6))
        words = [bytes(r) for r in cold] + [b"zzzzzz"] * 300_000 + [b"aaaaaa"] * 100_000 + [b"mmmmmm"] * 17
        order = rng.permutation(len(words))
        data = b"\n".join(words[i] for i in order)
    elif case == "hot_and_cold_wide":
        words = []
        for L in (12, 24):
            alpha = np.frombuffer(b"abcdefghijklmnopqrstuvwxyzABC", np.uint8)
            hot = [bytes(rng.choice(alpha, size=L)) for _ in range(5)]
            cold = rng.choice(alpha, size=(120_000, L))
            words += [bytes(r) for r in cold] + [hot[i] for i in rng.integers(0, 5, size=80_000)]
        order = rng.permutation(len(words))
        data = b" ".join(words[i] for i in order)
    else:
        lens = rng.integers(33, 37, size=60_000)  # four buckets of about 15,000 words
        words = [bytes(rng.choice(np.frombuffer(b"abcdefghijklmnopqrstuvwxyz", np.uint8), size=L)) for L in lens]
        data = b" ".join(words + words[:5_000])
    assert_same(ctx.text(data), oracle_mod.stable(data, nthreads=8), case)
