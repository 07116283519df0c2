"""The C-ABI library: builds, loads and exports every entry point that
include/bsort.h declares.  No compute calls (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bsort.h")


def declared_functions() -> list[str]:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bsort_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1407_6603_gb300 as bs

    return bs.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bsort_create", "bsort_text", "bsort_text_device", "bsort_batch", "bsort_destroy",
                     "bsort_result_release", "bsort_last_error", "bsort_config_default"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_library_is_built_for_sm_103a(libpath):
    objs = [os.path.join(os.path.dirname(libpath), f) for f in os.listdir(os.path.dirname(libpath)) if f.endswith(".o")]
    assert objs
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    assert "sm_103a" in out.stdout


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1407_6603_gb300 as bs

    with pytest.raises(RuntimeError, match="not found"):
        bs.load(str(tmp_path / "libbsort.so"))


def test_create_without_device_reports_cuda_error(libpath):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1407_6603_gb300 as bs

    with pytest.raises(bs.BsortError) as e:
        bs.bsort_create()
    assert e.value.status == bs.BSORT_E_CUDA


def test_config_default(libpath):
    import paper_1407_6603_gb300 as bs

    cfg = bs.bsort_config_default()
    assert cfg.l_cap == 255 and cfg.want_offsets == 1 and cfg.device == -1 and cfg.wait_limit == 0


def test_config_default_has_builtin_tuning(libpath):
    import paper_1407_6603_gb300 as bs

    assert bs.bsort_config_default().tune_table is None


@pytest.mark.parametrize("table", [
    "k4_lanes=3,4,4,4",        # lanes must be 2, 4 or 8
    "k4_lanes=4,4,4",          # one value per cluster size
    "k4_lanes=4,4,4,4,4",
    "piped_min=0",             # at least one tile per CTA
    "piped_min=-1",
    "piped_min=x",
    "bogus=1",                 # unknown key
    "k4_lanes",                # no value
    "k4_lanes=4,,4,4",
    "k4_runs=3",               # runs of 1, 2, 4 or 8 tiles
    "k4_streams=2",
    "k4_runs_small=4",         # 8 or 16
    "k4_threads=128,256,256,256",  # 256 or 512
])
def test_bad_tune_table_is_rejected_before_any_device_call(libpath, table):
    import paper_1407_6603_gb300 as bs

    cfg = bs.bsort_config_default()
    buf = table.encode()
    cfg.tune_table = buf
    with pytest.raises(bs.BsortError) as e:
        bs.bsort_create(cfg)
    assert e.value.status == bs.BSORT_E_INVAL


@pytest.mark.parametrize("table", ["", "# only a comment\n", "k4_lanes=2,4,8,8; piped_min=3", "k4_runs=1 k4_streams=0",
                                   "k4_lanes=8,8,8,8\npiped_min=1000000  # forced off\n"])
def test_good_tune_table_passes_the_parser(libpath, table):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1407_6603_gb300 as bs

    cfg = bs.bsort_config_default()
    buf = table.encode()
    cfg.tune_table = buf
    with pytest.raises(bs.BsortError) as e:  # parsed, then fails for want of a device
        bs.bsort_create(cfg)
    assert e.value.status == bs.BSORT_E_CUDA
