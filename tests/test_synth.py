"""The input generator: deterministic across hosts, and shaped as its recipe
says (sizes, separators, capitalisation and punctuation rates, Zipf draw)."""
import hashlib
import json
import os
import re

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "digests.json")


def _sha(b):
    return hashlib.sha256(bytes(b)).hexdigest()


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["plain_190k", "plain_1m38"])
def test_plain_digest(synth_mod, golden, name):
    d = synth_mod.plain(name)
    assert d.size == synth_mod.PLAIN[name].nbytes
    assert _sha(d) == golden["inputs"][name]


@pytest.mark.slow
def test_plain_256m_digest(synth_mod, golden):
    d = synth_mod.plain("plain_256m")
    assert d.size == 1 << 28
    assert _sha(d) == golden["inputs"]["plain_256m"]


def test_batch_shapes_and_digests(synth_mod, golden):
    shapes = synth_mod.batch_shapes(16)
    for (seed, n, v), g in zip(shapes, golden["batch_first16"]):
        assert (seed, n, v) == (g["seed"], g["nbytes"], g["vocab"])
        assert 1024 <= n <= 4 << 20 and 500 <= v <= 100_000
        assert _sha(synth_mod.batch_doc(seed, n, v)) == g["sha256"]


def test_batch_sizes_log_uniform(synth_mod):
    n = np.array([s[1] for s in synth_mod.batch_shapes(4096)], dtype=np.float64)
    logs = (np.log(n) - np.log(1024)) / (np.log(4 << 20) - np.log(1024))
    assert logs.min() >= 0 and logs.max() <= 1
    # uniform on [0,1]: mean 1/2, variance 1/12
    assert abs(logs.mean() - 0.5) < 0.02 and abs(logs.var() - 1 / 12) < 0.01


def test_recipe_statistics(synth_mod):
    c = synth_mod.PLAIN["plain_1m38"]
    d = bytes(synth_mod.plain("plain_1m38"))
    assert set(d) <= set(b"abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ ,.;:?!\"'-\n")
    assert "  " not in d.decode() and "\n\n" not in d.decode()
    lines = d.split(b"\n")[:-1]  # the last line is cut by the byte budget
    per_line = [len(line.split(b" ")) for line in lines]
    assert min(per_line) >= 10 and max(per_line) <= 14
    assert set(per_line) == set(range(10, 15))
    toks = d.split()[:-1]
    cap = np.mean([t[0:1].isupper() for t in toks])
    punct = np.mean([t[-1:] in b",.;:?!\"'-" for t in toks])
    assert abs(cap - 0.12) < 0.01 and abs(punct - 0.10) < 0.01
    words = [re.sub(rb"[^a-z]", b"", t.lower()) for t in toks]
    assert all(1 <= len(w) <= c.lmax for w in words)
    vocab, freq = np.unique(np.array(words, dtype=object), return_counts=True)
    assert len(vocab) <= c.vocab
    # Zipf(1.07): log frequency against log rank over the top 200 ranks
    f = np.sort(freq)[::-1][:200].astype(np.float64)
    slope = np.polyfit(np.log(np.arange(1, 201)), np.log(f), 1)[0]
    assert -1.2 < slope < -0.95


def test_different_seeds_differ(synth_mod):
    a = synth_mod.text(synth_mod.TAG_PLAIN, 10, 5000, 300, 3.7, 20)
    b = synth_mod.text(synth_mod.TAG_PLAIN, 11, 5000, 300, 3.7, 20)
    c = synth_mod.text(synth_mod.TAG_PLAIN, 10, 5000, 300, 3.7, 20)
    assert bytes(a) != bytes(b) and bytes(a) == bytes(c)
