"""The oracle against its pins (hand-worked cases, brute force, invariants,
bubble-sort counting facts) and O1 == O2 on generated text."""
import numpy as np
import pytest

import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(oracle_mod, pin):
    pin(oracle_mod._load())


def test_bubble_equals_stable_on_plain_190k(oracle_mod, synth_mod):
    data = synth_mod.plain("plain_190k")
    a = oracle_mod.bubble(data, nthreads=8)
    b = oracle_mod.stable(data, nthreads=8)
    for k in ("counts", "offsets", "stream"):
        assert np.array_equal(a[k], b[k])
    oracle_pins.check_invariants(bytes(data), b)
    # the workload's recipe: ~32k words, lengths clipped to [1, 20]
    assert 25_000 < a["n_words"] < 40_000 and a["max_len"] <= 20


def test_tokenize_matches_python_split(oracle_mod, synth_mod):
    data = bytes(synth_mod.plain("plain_190k")[:50_000])
    assert oracle_mod.tokenize(data) == oracle_pins.python_tokens(data)
