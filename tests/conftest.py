import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def synth_mod():
    import synth

    synth.build()
    return synth


@pytest.fixture(scope="session")
def bsort_gpu():
    """The CUDA boundary, for tests marked gpu.  Fails (does not skip) when the
    library or the GPU is missing: a gpu test must never pass on a fallback."""
    import torch

    import paper_1407_6603_gb300 as bs

    assert torch.cuda.is_available(), "gpu test run without a CUDA device"
    bs.load()
    return bs
