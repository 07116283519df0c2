"""The autotuner's selection logic and its output, on the host: the timings
are replaced by a cost model with a known optimum, so the test checks that
each step picks what its timings favour and that the table it writes (and
the one shipped beside the library) is accepted by the library's parser."""
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the optimum of the cost model below
BEST = {"lanes": (2, 4, 2, 8), "threads": "512,512,512,256", "runs": 4, "runs_small": 16, "piped": 2}


def _parse(table: str) -> dict:
    out = {}
    for tok in table.split():
        k, v = tok.split("=")
        out[k] = v
    return out


def _fake_time(table, sets, reps):
    """(per-launch times per (family, variant), whole-call span) for a table."""
    t = _parse(table)
    lanes = tuple(int(x) for x in t.get("k4_lanes", "2,2,2,2").split(","))
    per = {}
    for i, cl in enumerate((1, 2, 4, 8)):  # each class alone: fastest at its BEST lane count
        per[("tile_sort", cl)] = reps * (1.0 + abs(lanes[i] - BEST["lanes"][i]))
    span = sum(abs(a - b) for a, b in zip(lanes, BEST["lanes"]))
    span += 0 if t.get("k4_threads", "256,256,256,256") == BEST["threads"] else 1
    span += abs(int(t.get("k4_runs", 1)) - BEST["runs"]) * (2 if len(sets) > 1 else 0)
    span += 0 if int(t.get("k4_runs_small", 8)) == BEST["runs_small"] else 1
    span += abs(int(t.get("piped_min", 1)) - BEST["piped"]) * (3 if len(sets) > 1 else 0)
    return per, reps * (10.0 + span)


@pytest.fixture()
def tuned(monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_1407_6603_gb300 import autotune

    # one small set; the run length and the threshold are only visible with
    # the large set added, as on the GPU
    monkeypatch.setattr(autotune, "_documents", lambda: ([("small", [])], [("large", [])]))
    monkeypatch.setattr(autotune, "_time", _fake_time)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "test device")
    return autotune.tune(reps=2, log=lambda *a: None)


def test_tuner_picks_what_its_timings_favour(tuned):
    lines = [ln for ln in tuned.splitlines() if ln and not ln.startswith("#")]
    got = dict(ln.split("=") for ln in lines)
    assert got["k4_lanes"] == ",".join(map(str, BEST["lanes"]))
    assert got["k4_threads"] == BEST["threads"]
    assert got["k4_runs"] == str(BEST["runs"])
    assert got["k4_runs_small"] == str(BEST["runs_small"])
    assert got["piped_min"] == str(BEST["piped"])
    assert "test device" in tuned.splitlines()[0]


def _assert_parses(table: str):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1407_6603_gb300 as bs

    cfg = bs.bsort_config_default()
    buf = table.encode()
    cfg.tune_table = buf
    with pytest.raises(bs.BsortError) as e:  # parsed, then fails for want of a device
        bs.bsort_create(cfg)
    assert e.value.status == bs.BSORT_E_CUDA, "the library rejected the table"


def test_tuner_output_passes_the_parser(tuned):
    _assert_parses(tuned)


def test_shipped_tune_table_passes_the_parser():
    with open(os.path.join(ROOT, "paper_1407_6603_gb300", "tune_table.txt")) as f:
        _assert_parses(f.read())


def test_shipped_table_is_the_built_in_tuning():
    """The library's built-in tuning (the Tune defaults in bsort_api.cu) is
    the table shipped beside it."""
    import re

    src = open(os.path.join(ROOT, "paper_1407_6603_gb300", "csrc", "bsort_api.cu")).read()
    body = src[src.index("struct Tune {"):src.index("\n};", src.index("struct Tune {"))]
    built_in = {}
    for key in ("k4_lanes", "k4_threads"):
        built_in[key] = ",".join(re.search(key + r"\[4\] = \{([^}]*)\}", body).group(1).replace(" ", "").split(","))
    for key in ("piped_min", "k4_runs", "k4_runs_small", "k4_streams"):
        built_in[key] = re.search(r"\b" + key + r" = (\d+);", body).group(1)
    with open(os.path.join(ROOT, "paper_1407_6603_gb300", "tune_table.txt")) as f:
        shipped = dict(ln.strip().split("=") for ln in f if ln.strip() and not ln.startswith("#"))
    for key, value in shipped.items():
        assert built_in[key] == value, (key, built_in[key], value)
