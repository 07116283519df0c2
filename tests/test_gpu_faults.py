"""Failure detection without a GPU fault.

* Bounded device waits: a context whose wait limit is far too small for the
  decoupled look-back of the tokenize kernel and the grid barriers of the
  merge passes gives up those waits.  Every call must then return
  BSORT_E_TIMEOUT or the oracle's exact result, never a wrong BSORT_OK, and
  the GPU context must stay usable (a default context afterwards is exact).
* Host-side injection (the environment variable BSORT_FAULT): allocation
  failures give BSORT_E_NOMEM, injected timeouts BSORT_E_TIMEOUT, and the
  context works again once the injection is cleared.
* Serving: admission under a budget that fits about one document with two
  workers (every tag comes back exactly once), and a batch that fails as a
  whole while it holds an empty document.
"""
import os
import threading
import time

import numpy as np
import pytest

from test_gpu_parity import assert_same, assert_same_dev

pytestmark = pytest.mark.gpu


@pytest.fixture
def fault_env():
    """Sets BSORT_FAULT for the test and always clears it afterwards."""
    def set_(v):
        if v:
            os.environ["BSORT_FAULT"] = v
        else:
            os.environ.pop("BSORT_FAULT", None)

    yield set_
    os.environ.pop("BSORT_FAULT", None)


def _doc(synth_mod, nbytes, seed):
    return synth_mod.text(synth_mod.TAG_FUZZ, seed, nbytes, 3_000, 3.7, 20)


def test_small_wait_limit_gives_timeout_or_exact(bsort_gpu, oracle_mod, synth_mod):
    import torch

    data = _doc(synth_mod, 3 << 20, 501)  # 192 chunks of K1; buckets that need merge passes
    exp = oracle_mod.stable(data, nthreads=8)
    outcomes = []
    for limit, tune in ((1, None), (2, None), (16, "dedupe=2"), (256, None), (256, "dedupe=2"), (4096, "dedupe=2")):
        # (dedupe=2: the duplicate-aware sort, whose hash inserts wait on each other)
        with bsort_gpu.Context(wait_limit=limit, tune_table=tune) as c:
            for _ in range(2):  # the same context twice: it stays usable after a timeout
                try:
                    r = c.text(data)
                except bsort_gpu.BsortError as e:
                    assert e.status == bsort_gpu.BSORT_E_TIMEOUT, str(e)
                    outcomes.append("timeout")
                    continue
                assert_same(r, exp, f"wait_limit={limit}")
                outcomes.append("ok")
            # the device entry point: K1's timeout in the call, the sort
            # kernels' through bsort_device_finish
            d_in = torch.from_numpy(data).cuda()
            try:
                dev = c.text_device(d_in)
            except bsort_gpu.BsortError as e:
                assert e.status == bsort_gpu.BSORT_E_TIMEOUT, str(e)
                outcomes.append("timeout")
            else:
                st = c.device_finish()
                assert st in (bsort_gpu.BSORT_OK, bsort_gpu.BSORT_E_TIMEOUT)
                if st == bsort_gpu.BSORT_OK:
                    assert_same_dev(dev, exp, f"device, wait_limit={limit}")
                outcomes.append("ok" if st == bsort_gpu.BSORT_OK else "timeout")
    # a wait limit of one poll cannot cover 192 chunks' look-back
    assert "timeout" in outcomes
    with bsort_gpu.Context() as c:
        assert_same(c.text(data), exp, "default context after the timeouts")
        dev = c.text_device(torch.from_numpy(data).cuda())
        assert c.device_finish() == bsort_gpu.BSORT_OK
        assert_same_dev(dev, exp, "default context, device entry point")


def test_injected_allocation_failure(bsort_gpu, oracle_mod, synth_mod, fault_env):
    data = _doc(synth_mod, 200_000, 502)
    exp = oracle_mod.stable(data)
    fault_env("alloc")
    with pytest.raises(bsort_gpu.BsortError) as ei:
        bsort_gpu.Context()
    assert ei.value.status == bsort_gpu.BSORT_E_NOMEM
    fault_env(None)
    with bsort_gpu.Context() as c:
        fault_env("alloc")
        with pytest.raises(bsort_gpu.BsortError) as ei:
            c.text(data)  # a fresh context must grow its buffers: fails
        assert ei.value.status == bsort_gpu.BSORT_E_NOMEM
        assert "BSORT_FAULT" in c.last_error()
        st, rs = c.batch([data, b"", data[:1000]])
        assert st == bsort_gpu.BSORT_E_NOMEM
        fault_env(None)
        assert_same(c.text(data), exp, "after the injected failure")
        fault_env("alloc")
        # buffers are large enough now: a call that needs no allocation works
        assert_same(c.text(data), exp, "no allocation needed")


def test_injected_timeout(bsort_gpu, oracle_mod, synth_mod, fault_env):
    data = _doc(synth_mod, 100_000, 503)
    exp = oracle_mod.stable(data)
    with bsort_gpu.Context() as c:
        fault_env("timeout")
        with pytest.raises(bsort_gpu.BsortError) as ei:
            c.text(data)
        assert ei.value.status == bsort_gpu.BSORT_E_TIMEOUT
        fault_env(None)
        assert_same(c.text(data), exp)


def _serve_collect(c, n, timeout_s=120):
    got = {}
    deadline = time.time() + timeout_s
    while len(got) < n and time.time() < deadline:
        for tag, res, _ in c.poll(16):
            assert tag not in got, f"tag {tag} returned twice"
            got[tag] = res
        time.sleep(0.001)
    return got


def test_serving_tight_budget_two_workers(bsort_gpu, oracle_mod, synth_mod):
    """A budget that fits about one document: the two workers take turns at
    the queue front while waiting for budget; every tag comes back exactly
    once with the oracle's result."""
    docs = [_doc(synth_mod, 60_000 + 7_000 * i, 600 + i) for i in range(16)]
    foot = 16 * max(d.size for d in docs) + (64 << 10)  # the server's per-document footprint
    with bsort_gpu.Context() as c:
        c.serve_start(hbm_budget=foot + foot // 2, workers=2, max_batch_docs=4)

        def producer():
            for i, d in enumerate(docs):
                assert c.submit(d, i) == 0
                if i % 3 == 0:
                    time.sleep(0.002)

        th = threading.Thread(target=producer)
        th.start()
        got = _serve_collect(c, len(docs))
        th.join()
        c.serve_stop()
    assert sorted(got) == list(range(len(docs)))
    for i, d in enumerate(docs):
        assert got[i].status == 0
        assert_same(got[i], oracle_mod.stable(d, nthreads=8), f"request {i}")


def test_serving_failed_batch_with_empty_document(bsort_gpu, oracle_mod, fault_env):
    """A batch whose call fails as a whole (allocation failure injected in the
    workers' fresh contexts) while it holds an empty document: every request
    comes back with the call's status, and the server works afterwards."""
    docs = [b"", b"several words in here", b""]
    with bsort_gpu.Context() as c:
        c.serve_start(hbm_budget=1 << 30, workers=1, max_batch_docs=8)
        fault_env("alloc")
        for i, d in enumerate(docs):
            assert c.submit(d, i) == 0
        got = _serve_collect(c, len(docs))
        fault_env(None)
        assert sorted(got) == [0, 1, 2]
        assert all(got[i].status == bsort_gpu.BSORT_E_NOMEM for i in range(3))
        for i, d in enumerate(docs):
            assert c.submit(d, 10 + i) == 0
        again = _serve_collect(c, len(docs))
        c.serve_stop()
    assert sorted(again) == [10, 11, 12]
    for i, d in enumerate(docs):
        assert again[10 + i].status == 0
        assert_same(again[10 + i], oracle_mod.stable(d), f"request {10 + i}")
