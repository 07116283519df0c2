"""Pins for the oracle: checks against what the paper and plain mathematics
fix, never against the oracle itself.

Each ``pin_*`` function takes a loaded oracle library (``oracle.bind(path)``)
and raises AssertionError on a mismatch.  ``tests/test_oracle_pins.py`` runs
them on the real oracle; ``tests/test_oracle_mutants.py`` runs them on copies
of the oracle with a planted mistake and requires that some pin fails.

Sources of truth used here:
  * hand-worked examples, derived step by step in the comments from the
    paper's three pre-processing phases (Section II) and its description of
    bubble sort (Section I);
  * Python's own ``sorted`` with key (length, bytes) and ``str.split`` style
    whitespace splitting: library routines the definition reduces to;
  * brute force: every permutation of a small word multiset gives the same
    output (the result is unique);
  * bubble sort facts: swaps = inversions, comparisons = n(n-1)/2 on a
    reversed bucket (the cost the paper states in "Bubble sort as parallel")
    and n-1 on a sorted one (early exit).
"""
from __future__ import annotations

import itertools
import random

import numpy as np

import oracle

WS = b" \t\n\x0b\x0c\r"


def _words(res) -> list[bytes]:
    return oracle.words_of(res)


def python_tokens(data: bytes) -> list[bytes]:
    """Independent tokenizer: split on C-locale whitespace (bytes.split() uses
    exactly 0x20 and 0x09-0x0D), keep ASCII letters, drop empty words."""
    out = []
    for field in data.split():
        w = bytes(c for c in field if (65 <= c <= 90) or (97 <= c <= 122))
        if w:
            out.append(w)
    return out


def python_sorted(tokens: list[bytes]) -> list[bytes]:
    return sorted(tokens, key=lambda w: (len(w), w))


def check_invariants(data: bytes, res: dict) -> None:
    toks = python_tokens(data)
    words = _words(res)
    assert res["n_words"] == len(toks) == len(words)
    assert sorted(words) == sorted(toks), "output is not a permutation of the stripped words"
    lens = [len(w) for w in words]
    assert lens == sorted(lens), "lengths must be non-decreasing"
    for a, b in zip(words, words[1:]):
        if len(a) == len(b):
            assert a <= b, "each bucket must be in unsigned byte order"
    counts = np.asarray(res["counts"]).tolist()
    assert counts[0] == 0
    assert sum(counts) == len(toks)
    assert sum(L * c for L, c in enumerate(counts)) == res["stream_bytes"] == sum(lens)
    assert res["max_len"] == (max(lens) if lens else 0)
    assert len(counts) == res["max_len"] + 1
    if lens:
        assert counts[-1] > 0
    off = np.asarray(res["offsets"]).tolist()
    assert off[0] == 0 and off[-1] == res["stream_bytes"]
    assert all(off[i + 1] - off[i] == lens[i] for i in range(len(lens)))
    assert words == python_sorted(toks)


def _both(lib, data, nthreads=1):
    return (oracle.bubble(data, nthreads, lib=lib), oracle.stable(data, nthreads, lib=lib))


def pin_hand_example(lib):
    # Input:  "Hello, world! The cat-sat\non a mat; The end."
    # Phase 1 (strip): punctuation is deleted, '-' inside "cat-sat" joins it,
    #   whitespace splits: Hello world The catsat on a mat The end   (9 words)
    # Phase 2 (bucket by length): L=1 [a]  L=2 [on]  L=3 [The mat The end]
    #   L=4 []  L=5 [Hello world]  L=6 [catsat]
    # Phase 3 (ASCII order; 'T'=84 < 'e'=101 < 'm'=109):
    #   L=3 -> The The end mat ; L=5 -> Hello ('H'=72) world ('w'=119)
    data = b"Hello, world! The cat-sat\non a mat; The end."
    for res in _both(lib, data):
        assert res["max_len"] == 6
        assert res["n_words"] == 9
        assert np.asarray(res["counts"]).tolist() == [0, 1, 1, 4, 0, 2, 1]
        assert bytes(res["stream"]) == b"aonTheTheendmatHelloworldcatsat"
        assert np.asarray(res["offsets"]).tolist() == [0, 1, 3, 6, 9, 12, 15, 20, 25, 31]
    # Bubble sort on bucket L=3 [The mat The end]:
    #   pass 0: (The,mat) keep; (mat,The) swap; (mat,end) swap -> The The end mat
    #   pass 1: (The,The) keep; (The,end) keep -> no swap, stop.
    # L=5 [Hello world]: one comparison, no swap.  Total 3+2+1 = 6 comparisons, 2 swaps.
    res = oracle.bubble(data, 1, lib=lib)
    assert res["compares"] == 6 and res["swaps"] == 2


def pin_special_cases(lib):
    cases = {
        b"": [],
        b"!!! ... ---": [],                          # nothing but special characters
        b" \t\n\x0b\x0c\r ": [],                      # every whitespace byte
        b"a\tb\r\nc": [b"a", b"b", b"c"],            # tab, CR, LF all separate
        b"a\x0bb\x0cc": [b"a", b"b", b"c"],          # VT and FF separate too
        b"\xc3\xa9t\xc3\xa9": [b"t"],                # UTF-8 bytes are not letters
        b"don't can't": [b"cant", b"dont"],         # apostrophe deleted, not a split
        b"abc123 456": [b"abc"],                     # digits are special characters
        b"a\x00b": [b"ab"],                          # NUL is not whitespace
        b"Zebra apple": [b"Zebra", b"apple"],        # 'Z'=90 < 'a'=97
        b"b a b a": [b"a", b"a", b"b", b"b"],        # duplicates kept
        b"zz y xxx": [b"y", b"zz", b"xxx"],          # shorter buckets first
        b"@@@ a": [b"a"],                            # field with no letters dropped
        b"x" * 300: [b"x" * 300],                    # one long word
        b"q": [b"q"],
        b"ab-\n-cd": [b"ab", b"cd"],                 # punctuation at both ends
    }
    for data, expect in cases.items():
        for res in _both(lib, data):
            assert _words(res) == expect, (data, _words(res))
            check_invariants(data, res)
    empty = oracle.bubble(b"", 1, lib=lib)
    assert empty["max_len"] == 0 and np.asarray(empty["counts"]).tolist() == [0]
    assert np.asarray(empty["offsets"]).tolist() == [0]


def pin_brute_force_permutations(lib):
    # Every order of the same words gives one output: the result is unique,
    # and it equals Python's sorted() by (length, bytes).
    rng = random.Random(1234)
    multisets = [
        [b"A", b"a", b"b", b"ab", b"ba", b"Ab", b"a"],
        [b"ba", b"ab", b"Ab", b"aB", b"BA", b"b"],
        [b"abc", b"abd", b"ab", b"a", b"abc", b"Abc"],
    ]
    for ms in multisets:
        expect = python_sorted(ms)
        seen = set()
        for perm in itertools.permutations(range(len(ms))):
            parts = []
            for i in perm:
                w = ms[i]
                # decorate with punctuation inside/around and random whitespace
                if rng.random() < 0.3:
                    cut = rng.randrange(len(w) + 1)
                    w = w[:cut] + bytes([rng.choice(b"-'.,!?\"")]) + w[cut:]
                parts.append(w)
                parts.append(bytes([rng.choice(WS)]) * rng.randint(1, 2))
            data = b"".join(parts)
            if len(seen) < 2:
                seen.add(data)
            res = oracle.bubble(data, 1, lib=lib)
            assert _words(res) == expect, (data, _words(res))
        res2 = oracle.stable(data, 1, lib=lib)
        assert _words(res2) == expect


def _fuzz_doc(rng: random.Random, n: int) -> bytes:
    alphabet = (b"abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ" * 3 + WS * 4 + b".,;:?!\"'-0123456789"
                + bytes(range(128, 256, 7)) + b"\x00\x01\x7f")
    return bytes(rng.choice(alphabet) for _ in range(n))


def pin_invariants_fuzz(lib):
    rng = random.Random(99)
    for trial in range(60):
        data = _fuzz_doc(rng, rng.randint(0, 3000))
        a, b = _both(lib, data, nthreads=1 + trial % 4)
        check_invariants(data, a)
        check_invariants(data, b)
        for k in ("counts", "offsets", "stream"):
            assert np.array_equal(a[k], b[k])


def _inversions(seq: list[bytes]) -> int:
    return sum(1 for i in range(len(seq)) for j in range(i + 1, len(seq)) if seq[i] > seq[j])


def pin_bubble_counts(lib):
    rng = random.Random(7)
    # swaps == inversions of each bucket in input order; comparisons bounded
    # by n(n-1)/2 per bucket.
    for _ in range(15):
        words = [bytes(rng.choice(b"abcAB") for _ in range(rng.randint(1, 4))) for _ in range(rng.randint(0, 80))]
        data = b" ".join(words)
        res = oracle.bubble(data, 2, lib=lib)
        toks = python_tokens(data)
        by_len: dict[int, list[bytes]] = {}
        for t in toks:
            by_len.setdefault(len(t), []).append(t)
        assert res["swaps"] == sum(_inversions(v) for v in by_len.values())
        assert res["compares"] <= sum(len(v) * (len(v) - 1) // 2 for v in by_len.values())
    # A bucket in reverse order costs exactly n(n-1)/2 comparisons and swaps.
    for n in (1, 2, 3, 10, 57):
        words = sorted({bytes([97 + i // 26, 97 + i % 26]) for i in range(n)}, reverse=True)
        res = oracle.bubble(b" ".join(words), 1, lib=lib)
        assert res["compares"] == n * (n - 1) // 2 and res["swaps"] == n * (n - 1) // 2
        # already sorted: one pass of n-1 comparisons, then stop
        res = oracle.bubble(b"\n".join(reversed(words)), 1, lib=lib)
        assert res["compares"] == max(n - 1, 0) and res["swaps"] == 0


def pin_thread_count_invariance(lib):
    rng = random.Random(5)
    data = _fuzz_doc(rng, 20000)
    ref = oracle.bubble(data, 1, lib=lib)
    for t in (2, 3, 8):
        for res in _both(lib, data, nthreads=t):
            for k in ("counts", "offsets", "stream"):
                assert np.array_equal(ref[k], res[k])
    assert oracle.bubble(data, 4, lib=lib)["swaps"] == ref["swaps"]


# ---- the other orders (oracle.ORDER_*) ----
# References written from each order's definition with Python's own sort:
#   folded: (length, letters with case ignored, bytes);
#   whole:  the bytes alone (Python compares bytes lexicographically, a
#           prefix before its extensions);
#   length: the length alone, Python's sort being stable (input order kept).
ORDER_KEYS = {
    oracle.ORDER_ASCII: lambda w: (len(w), w),
    oracle.ORDER_FOLDED: lambda w: (len(w), w.lower(), w),
    oracle.ORDER_WHOLE: lambda w: w,
    oracle.ORDER_LENGTH: len,
}


def pin_orders_hand_example(lib):
    # Tokens of the example, in input order: Hello world The catsat on a mat
    # The end apple Apple APPLE aPple.  Worked by hand:
    #   folded: length 3 by case-blind letters: end < mat < the (The, The);
    #           length 5: the four spellings of "apple" first, among
    #           themselves in ASCII order (APPLE < Apple < aPple < apple),
    #           then Hello, world;
    #   whole:  upper-case letters before lower-case ones, a prefix first;
    #   length: each length keeps input order.
    data = b"Hello, world! The cat-sat\non a mat; The end. apple Apple APPLE aPple"
    want = {
        oracle.ORDER_FOLDED: [b"a", b"on", b"end", b"mat", b"The", b"The", b"APPLE", b"Apple", b"aPple", b"apple",
                              b"Hello", b"world", b"catsat"],
        oracle.ORDER_WHOLE: [b"APPLE", b"Apple", b"Hello", b"The", b"The", b"a", b"aPple", b"apple", b"catsat", b"end",
                             b"mat", b"on", b"world"],
        oracle.ORDER_LENGTH: [b"a", b"on", b"The", b"mat", b"The", b"end", b"Hello", b"world", b"apple", b"Apple",
                              b"APPLE", b"aPple", b"catsat"],
    }
    for order, words in want.items():
        for res in (oracle.bubble_order(data, order, 1, lib=lib), oracle.stable_order(data, order, 1, lib=lib)):
            assert _words(res) == words, (order, _words(res))
            assert res["counts"].tolist() == [0, 1, 1, 4, 0, 6, 1]
    # a prefix comes before its extensions; case is not folded in the whole order
    res = oracle.stable_order(b"abc ab b a ba B", oracle.ORDER_WHOLE, 1, lib=lib)
    assert _words(res) == [b"B", b"a", b"ab", b"abc", b"b", b"ba"]


def pin_orders_vs_python(lib):
    rng = random.Random(11)
    for trial in range(6):
        data = _fuzz_doc(rng, 3000 if trial < 3 else 400)
        toks = python_tokens(data)
        for order, key in ORDER_KEYS.items():
            want = sorted(toks, key=key)
            got = _words(oracle.stable_order(data, order, 2, lib=lib))
            assert got == want, (order, trial)
            if trial >= 3:  # bubble sort of the whole text is quadratic: small documents only
                assert _words(oracle.bubble_order(data, order, 2, lib=lib)) == want, (order, trial)
        assert _words(oracle.stable_order(data, oracle.ORDER_ASCII, 1, lib=lib)) == _words(oracle.stable(data, 1, lib=lib))


def pin_orders_brute_force(lib):
    # Every order of a small multiset with case variants: the sorted orders
    # give one result whatever the input order; the length order gives the
    # input order within each length.
    base = [b"ab", b"Ab", b"aB", b"a", b"B", b"ba", b"abc"]
    for perm in itertools.permutations(base):
        data = b" ".join(perm)
        for order, key in ORDER_KEYS.items():
            got = _words(oracle.bubble_order(data, order, 1, lib=lib))
            assert got == sorted(perm, key=key), (order, perm)
            assert got == _words(oracle.stable_order(data, order, 1, lib=lib))


ALL_PINS = [
    pin_orders_hand_example,
    pin_orders_vs_python,
    pin_orders_brute_force,
    pin_hand_example,
    pin_special_cases,
    pin_brute_force_permutations,
    pin_invariants_fuzz,
    pin_bubble_counts,
    pin_thread_count_invariance,
]
