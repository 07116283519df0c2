"""Every setting the autotuner can choose gives the oracle's result: the
odd-even/merge cutoff of each tile-sort class (2, 4 or 8 lanes per group), the
run length the tile sort leaves for the merge passes (clusters of 1, 2, 4, 8),
the side streams and the pipelined-merge threshold (always on, never on)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def assert_same(got, exp, label=""):
    assert got.n_words == exp["n_words"], label
    assert got.max_len == exp["max_len"], label
    assert np.array_equal(got.counts, exp["counts"]), label
    assert np.array_equal(got.offsets, exp["offsets"]), label
    assert np.array_equal(got.stream, exp["stream"]), label

TABLES = ["k4_lanes=2,2,2,2 piped_min=1 dedupe=0", "k4_lanes=8,8,8,8 piped_min=1000000 dedupe=0",
          "k4_lanes=2,8,4,2 piped_min=1 dedupe=0", "k4_lanes=8,4,2,8 piped_min=4 dedupe=0",
          "k4_runs=1 piped_min=1 dedupe=0", "k4_runs=2 k4_streams=0 dedupe=0", "k4_runs=4 dedupe=0",
          "k4_runs_small=16 dedupe=0", "k4_runs_small=16 k4_streams=0 k4_lanes=8,8,8,8",
          "k4_threads=512,512,512,512", "k4_threads=512,256,512,256 k4_lanes=8,2,2,4 k4_runs_small=16",
          "k4_runs=1 piped_min=1 dedupe=2", "k4_runs=8 k4_runs_small=8 dedupe=2", "k4_streams=0 dedupe=2"]


def threshold_doc(W):
    rng = np.random.default_rng(200 + W)
    kpt = 8 // W
    warp, tile = 32 * kpt, 2048 // W
    L = {1: 6, 2: 12, 4: 20}[W]
    words = []
    for n in (warp + 1, tile, 2 * tile + 1, 4 * tile + 1, 8 * tile + 1, 19 * tile + 3):
        letters = rng.choice(np.frombuffer(b"abAB", np.uint8), size=(n, L))
        words.extend(bytes(r) for r in letters)
    order = rng.permutation(len(words))
    return b" ".join(words[i] for i in order)


@pytest.mark.parametrize("table", TABLES)
def test_tuning_choices_agree_with_oracle(bsort_gpu, oracle_mod, synth_mod, table):
    docs = [synth_mod.plain("plain_1m38").tobytes(), threshold_doc(1), threshold_doc(2), threshold_doc(4)]
    with bsort_gpu.Context(tune_table=table) as c:
        for i, d in enumerate(docs):
            assert_same(c.text(d), oracle_mod.stable(d, nthreads=8), f"{table} doc {i}")


def test_tuning_applies_to_launches(bsort_gpu):
    """The trace shows the tile sorts' cluster sizes, and the merge threshold
    switches the pipelined merge (cut kernel) on and off."""
    rng = np.random.default_rng(11)
    n = 1_500_000  # one bucket of 1.5M five-letter words: about 730 merge tiles
    letters = rng.choice(np.frombuffer(b"abcdefgh", np.uint8), size=(n, 5))
    data = np.concatenate([letters, np.full((n, 1), 32, np.uint8)], axis=1).reshape(-1)
    cuts = {}
    for table in ("piped_min=1 dedupe=0", "piped_min=1000000 dedupe=0"):
        with bsort_gpu.Context(profile=1, tune_table=table) as c:
            c.profile_read()
            r = c.text(data)
            assert r.n_words == n
            tl = c.trace_read()
        assert {v[5] for v in tl if v[0] == "tile_sort"} <= {0, 1, 2, 4, 8, 16}
        cuts[table] = sum(1 for v in tl if v[0] == "merge_cut")
    assert cuts["piped_min=1 dedupe=0"] > 0 and cuts["piped_min=1000000 dedupe=0"] == 0
