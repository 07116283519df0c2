"""The other orders and key encodings on the GPU, against the oracle.

* key_pack=KEYS_LETTERS6: six-bit letter codes, ten letters to a key word;
  the result must be the ASCII order's, byte for byte.
* order=ORDER_FOLDED: alphabetic order with case ignored, ties in ASCII
  order, per length bucket; compared with the oracle's folded order.
* order=ORDER_WHOLE: every word of a document in ASCII order, a word before
  the longer words it begins (one bucket per document, zero-padded keys),
  with byte and six-bit keys.
* order=ORDER_LENGTH: length buckets in input order (no sort at all).
Each runs with the duplicate-aware sort forced on (dedupe=2) and off; the
whole and length orders never use it, so there both must agree anyway.
"""
import random

import numpy as np
import pytest

from test_gpu_parity import assert_same, assert_same_dev

pytestmark = pytest.mark.gpu

MODES = [("letters6", dict(key_pack=1), 0), ("folded", dict(order=1), 1), ("folded6", dict(order=1, key_pack=1), 1),
         ("whole", dict(order=2), 2), ("whole6", dict(order=2, key_pack=1), 2), ("length", dict(order=3), 3)]


@pytest.fixture(scope="module", params=[(m, t) for m in MODES for t in ("dedupe=2", "dedupe=0")],
                ids=lambda p: f"{p[0][0]}-{p[1]}")
def octx(bsort_gpu, request):
    (name, kw, order), tune = request.param
    c = bsort_gpu.Context(tune_table=tune, **kw)
    yield c, order
    c.close()


def expect(oracle_mod, data, order):
    return oracle_mod.stable_order(data, order, 8)


def case_mix(rng, n):
    """Words of every length 1..70 in mixed case (key words cross every
    letter-code boundary: 8 | 10 letters a word, 64 | 128 | 256 bits), with
    case variants of one spelling and shared prefixes."""
    words = []
    for _ in range(n):
        L = rng.choice([rng.randint(1, 12), rng.randint(1, 24), rng.randint(1, 70)])
        base = "".join(rng.choice("abcxyz") for _ in range(L))
        words.append("".join(ch.upper() if rng.random() < 0.3 else ch for ch in base).encode())
    return b" ".join(words)


def test_orders_hand_example(octx, oracle_mod):
    c, order = octx
    data = b"Hello, world! The cat-sat\non a mat; The end. apple Apple APPLE aPple zebra Zebra"
    assert_same(c.text(data), expect(oracle_mod, data, order))


@pytest.mark.parametrize("seed", [1, 2])
def test_orders_mixed_lengths_and_case(octx, oracle_mod, seed):
    c, order = octx
    data = case_mix(random.Random(seed), 20_000)
    assert_same(c.text(data), expect(oracle_mod, data, order))


def test_orders_every_length(octx, oracle_mod):
    c, order = octx
    rng = random.Random(3)
    words = []
    for L in range(1, 256):
        for _ in range(rng.randint(1, 12)):
            words.append(bytes(rng.choice(b"abcXYZ") for _ in range(L)))
    rng.shuffle(words)
    data = b" ".join(words)
    assert_same(c.text(data), expect(oracle_mod, data, order))


def test_orders_paper_sized_and_large_buckets(octx, oracle_mod, synth_mod):
    import torch

    c, order = octx
    for data in (synth_mod.plain("plain_1m38"), synth_mod.text(synth_mod.TAG_FUZZ, 91, 3 << 20, 3_000, 5.5, 40)):
        exp = expect(oracle_mod, data, order)
        assert_same(c.text(data), exp)
        assert_same_dev(c.text_device(torch.from_numpy(data).cuda()), exp)
        torch.cuda.synchronize()


def test_orders_batch(octx, oracle_mod, synth_mod):
    c, order = octx
    docs = [synth_mod.batch_doc(*s) for s in synth_mod.batch_shapes(20)]
    docs[2] = np.zeros(0, np.uint8)
    st, rs = c.batch(docs)
    assert st == 0
    for i, d in enumerate(docs):
        assert_same(rs[i], expect(oracle_mod, d, order), f"doc {i}")


def test_orders_prefixes_and_duplicates(octx, oracle_mod):
    """Words that begin other words, many copies of few spellings, and
    documents of one word or one length."""
    c, order = octx
    rng = random.Random(7)
    stems = [b"a", b"ab", b"abc", b"abcdefgh", b"abcdefghi", b"abcdefghij", b"abcdefghijk", b"B", b"Ba", b"z" * 17]
    words = [rng.choice(stems) + (b"" if rng.random() < 0.6 else bytes(rng.choice(b"aZ") for _ in range(rng.randint(1, 9))))
             for _ in range(30_000)]
    for data in (b" ".join(words), b"single", b"same same same SAME", b"abc abd abe ab a"):
        assert_same(c.text(data), expect(oracle_mod, data, order))


def test_letters6_is_the_ascii_result(bsort_gpu, synth_mod):
    """The six-bit keys change the keys, never the result."""
    data = synth_mod.plain("plain_190k")
    with bsort_gpu.Context() as a, bsort_gpu.Context(key_pack=1) as b:
        ra, rb = a.text(data), b.text(data)
        assert np.array_equal(ra.stream, rb.stream) and np.array_equal(ra.offsets, rb.offsets)


def test_bad_order_or_key_pack_is_rejected(bsort_gpu):
    for kw in (dict(order=9), dict(key_pack=7)):
        with pytest.raises(bsort_gpu.BsortError) as ei:
            bsort_gpu.Context(**kw)
        assert ei.value.status == bsort_gpu.BSORT_E_INVAL
