"""Kernel tracing through the C ABI: per-family statistics and the per-launch
timeline of a profiled call."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FAMILIES = {"tokenize", "layout", "scatter", "tile_sort", "merge_pass", "merge_cut", "emit", "host_gap", "expand",
            "dedupe"}


def test_profile_and_timeline(bsort_gpu, synth_mod):
    data = synth_mod.plain("plain_1m38")
    with bsort_gpu.Context(profile=1) as c:
        c.profile_read()
        n0 = c.launch_count()
        c.text(data)
        launches = c.launch_count() - n0
        tl = c.trace_read()
        stats = c.profile_read()
        assert c.trace_read() == []  # the profile read clears the records
    assert {r[0] for r in tl} <= FAMILIES
    # every kernel launch is traced (a record counts the kernels it covers),
    # plus the host round trip
    assert sum(r[6] for r in tl if r[0] != "host_gap") == launches
    assert all(r[6] >= 1 for r in tl if r[0] != "host_gap")
    assert sum(1 for r in tl if r[0] == "host_gap") == 1
    assert tl[0][0] == "tokenize" and tl[0][1] == 0.0
    # the bucket layout runs on the device, between the tokenizer and the round trip
    assert tl[1][0] == "layout" and tl[1][6] == 1  # one document: the one-CTA form
    for name, s, e, b, st, var, nk in tl:
        assert 0.0 <= s <= e, name
        assert 0 <= st <= 4
        if name == "tile_sort":
            assert var in (0, 1, 2, 4, 8, 16)  # CTAs per cluster, 0 for the warp sort
        if name in ("merge_pass", "merge_cut"):
            assert var in (1, 2, 4, 8, 16, 32)  # key width
    for name in {r[0] for r in tl}:
        ms = sum(e - s for n, s, e, *_ in tl if n == name)
        assert stats[name][1] == pytest.approx(ms, rel=1e-3, abs=1e-3), name
        # (a host gap is no kernel: its count is the number of gaps)
        want = sum(1 if name == "host_gap" else r[6] for r in tl if r[0] == name)
        assert stats[name][0] == want, name
    # the tokenizer runs first, every sort launch starts after the round trip
    gap = next(r for r in tl if r[0] == "host_gap")
    assert all(r[1] >= gap[1] for r in tl if r[0] in ("scatter", "tile_sort", "merge_pass"))
    lay = next(r for r in tl if r[0] == "layout")
    assert lay[2] <= gap[1] + 1e-3
