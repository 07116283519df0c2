"""The bucket layout built on the device (K2), against the oracle.

One CTA of the layout holds 16 documents: batches of 16 take the one-launch
form, 17 and more the three-launch form (per-CTA sums, a scan by the last
CTA, then the table).  Every tenth... every fourth document here is large,
with buckets big enough for the merge passes or the duplicate-aware sort
(more than eight K4 tiles of keys), so that the numbering that runs across
buckets and documents (first key word, merge tiles, merge samples,
supertiles, hash-aggregation units, hash-table, array and count words) is
exercised across CTAs, with each way the tune table can route those buckets.
"""
import random

import numpy as np
import pytest

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu


def words_doc(rng, spec, alphabet="abcd"):
    """A document of rng-shuffled words: spec is a list of (count, length)."""
    words = []
    for count, L in spec:
        words += ["".join(rng.choice(alphabet) for _ in range(L)) for _ in range(count)]
    rng.shuffle(words)
    return np.frombuffer(" ".join(words).encode(), np.uint8)


def layout_batch(ndocs, seed):
    rng = random.Random(seed)
    docs = []
    for i in range(ndocs):
        if i % 4 == 1:
            # one-word keys (20k > 8 x 2048), two-word keys (9k > 8 x 1024), and a
            # four-word bucket K4 finishes in clusters of 8
            spec = [(20000 + 97 * i, 4), (9000 + 31 * i, 11), (3000, 20), (50, 7)]
        elif i % 4 == 3:
            spec = [(rng.randint(1, 40), rng.randint(1, 30)) for _ in range(12)]
        else:
            spec = [(rng.randint(1, 300), rng.randint(1, 12)) for _ in range(5)]
        docs.append(words_doc(rng, spec, "abcd" if i % 2 else "abcdefghijklmnopqrstuvwxyzABC"))
    if ndocs > 6:
        docs[6] = np.zeros(0, np.uint8)  # an empty document among them
    return docs


TUNES = ["dedupe=2", "dedupe=0", "dedupe=0 k4_runs=1 piped_min=1", "dedupe=0 k4_runs_small=16 piped_min=1000000"]


@pytest.mark.parametrize("tune", TUNES)
@pytest.mark.parametrize("ndocs", [16, 17, 40])
def test_layout_across_ctas(bsort_gpu, oracle_mod, ndocs, tune):
    docs = layout_batch(ndocs, 100 + ndocs)
    with bsort_gpu.Context(tune_table=tune) as c:
        st, rs = c.batch(docs)
        assert st == 0, c.last_error()
        for i, d in enumerate(docs):
            assert_same(rs[i], oracle_mod.stable(d, nthreads=8), f"doc {i}")


def test_layout_whole_order_across_ctas(bsort_gpu, oracle_mod):
    """The whole-text order's one bucket per document, over 17 documents
    (three-launch form), large ones too (merge passes of zero-padded keys)."""
    docs = layout_batch(17, 7)
    with bsort_gpu.Context(order=2) as c:
        st, rs = c.batch(docs)
        assert st == 0, c.last_error()
        for i, d in enumerate(docs):
            assert_same(rs[i], oracle_mod.stable_order(d, 2, 8), f"doc {i}")


def test_layout_failing_document_in_second_cta(bsort_gpu, oracle_mod):
    """A document with a word too long sits in the layout's second CTA: it
    gets no buckets, the others are laid out around it."""
    docs = layout_batch(20, 3)
    docs[18] = np.frombuffer(b"ok " + b"x" * 300 + b" fine", np.uint8)
    with bsort_gpu.Context() as c:
        st, rs = c.batch(docs)
        assert st == bsort_gpu.BSORT_E_WORD_TOO_LONG
        for i, d in enumerate(docs):
            if i == 18:
                assert rs[i].status == bsort_gpu.BSORT_E_WORD_TOO_LONG
                continue
            assert_same(rs[i], oracle_mod.stable(d, nthreads=8), f"doc {i}")
