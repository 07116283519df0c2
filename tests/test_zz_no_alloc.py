"""The allocation-free strip + tokenize entry point (bsort_strip_noalloc).

It exists for callers that cannot call cudaMalloc (code running during CUDA
graph capture, plugins whose host framework owns all device memory).  What it
promises is the document's words in input order, so that list is compared
element by element with the CPU oracle's tokenizer (oracle.tokenize), and its
output must also agree with the existing entry point's: the same words, put
in (length, bytes) order, are exactly the stream, offsets and counts that
bsort_text_device returns for the same document.  Two calls in a row check
that the shared scratch array is cleared between calls.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(bs, d_in, torch):
    n = d_in.numel()
    letters = torch.empty(max(n, 1), dtype=torch.uint8, device=d_in.device)
    starts = torch.full((n // 2 + 2,), -1, dtype=torch.int32, device=d_in.device)
    totals = torch.full((3,), -1, dtype=torch.int32, device=d_in.device)
    stream = torch.cuda.current_stream(d_in.device)
    st = bs.bsort_strip_noalloc(d_in.data_ptr() if n else 0, n, stream.cuda_stream, letters.data_ptr(),
                                starts.data_ptr(), totals.data_ptr())
    assert st == bs.BSORT_OK
    torch.cuda.synchronize()
    n_words, n_letters, status = totals.cpu().tolist()
    assert status == 0
    s = starts[: n_words + 1].cpu().numpy().astype(np.int64)
    assert s[0] == 0 or n_words == 0
    assert s[n_words] == n_letters
    buf = letters[:n_letters].cpu().numpy().tobytes()
    return [buf[s[i]:s[i + 1]] for i in range(n_words)]


def _check_against_existing(bs, ctx, d_in, words):
    ref = ctx.text_device(d_in)
    import torch

    torch.cuda.synchronize()
    assert len(words) == ref["n_words"]
    lens = np.array([len(w) for w in words], dtype=np.int64)
    assert int(lens.sum()) == ref["stream_bytes"]
    counts = np.bincount(lens, minlength=ref["max_len"] + 1) if len(words) else np.zeros(1, np.int64)
    assert counts.tolist() == ref["counts"].cpu().tolist()
    ordered = sorted(words, key=lambda w: (len(w), w))
    assert b"".join(ordered) == ref["stream"].cpu().numpy().tobytes()
    off = np.concatenate([[0], np.cumsum([len(w) for w in ordered])]).astype(np.int64)
    assert off.tolist() == ref["offsets"].cpu().numpy().astype(np.int64).tolist()


def _check_against_oracle(oracle_mod, data, words):
    """The input-order word list, element by element, against the oracle's."""
    exp = oracle_mod.tokenize(np.ascontiguousarray(data))
    assert len(words) == len(exp)
    for i, (w, e) in enumerate(zip(words, exp)):
        assert w == e, f"word {i}: {w!r} != {e!r}"


def test_noalloc_matches_oracle_and_existing_entry_point_twice(bsort_gpu, oracle_mod, synth_mod):
    import torch

    docs = [synth_mod.plain("plain_1m38"), synth_mod.text(synth_mod.TAG_FUZZ, 77, 300_001, 2_000, 3.7, 20)]
    with bsort_gpu.Context() as ctx:
        for data in docs:  # two calls in a row on the same scratch
            d_in = torch.from_numpy(np.ascontiguousarray(data)).cuda()
            words = _noalloc(bsort_gpu, d_in, torch)
            _check_against_oracle(oracle_mod, data, words)
            _check_against_existing(bsort_gpu, ctx, d_in, words)


def test_noalloc_chunk_straddling_words(bsort_gpu, oracle_mod):
    """Words and runs of punctuation that straddle the 16 KiB chunks the
    kernel splits the document into, on both sides of each boundary."""
    import torch

    rng = np.random.default_rng(79)
    alphabet = np.frombuffer(b"abcXYZ,.'- \n\t", np.uint8)
    data = rng.choice(alphabet, size=5 * 16384 + 77)
    for k in range(1, 6):  # one long word across each chunk boundary
        data[k * 16384 - 40:k * 16384 + 40] = ord("q")
    d_in = torch.from_numpy(data).cuda()
    _check_against_oracle(oracle_mod, data, _noalloc(bsort_gpu, d_in, torch))


def test_noalloc_unaligned_and_empty(bsort_gpu, oracle_mod, synth_mod):
    import torch

    data = synth_mod.text(synth_mod.TAG_FUZZ, 78, 40_000, 500, 3.7, 20)
    buf = torch.zeros(data.size + 32, dtype=torch.uint8, device="cuda")
    buf[5:5 + data.size] = torch.from_numpy(data).cuda()
    with bsort_gpu.Context() as ctx:
        view = buf[5:5 + data.size]
        words = _noalloc(bsort_gpu, view, torch)
        _check_against_oracle(oracle_mod, data, words)
        _check_against_existing(bsort_gpu, ctx, view, words)
        empty = torch.zeros(0, dtype=torch.uint8, device="cuda")
        assert _noalloc(bsort_gpu, empty, torch) == []


def test_noalloc_rejects_documents_over_the_limit(bsort_gpu):
    import torch

    small = torch.zeros(16, dtype=torch.uint8, device="cuda")
    # rejected on the host before any GPU work: the buffers are never touched
    st = bsort_gpu.bsort_strip_noalloc(small.data_ptr(), bsort_gpu.NOALLOC_MAX_BYTES + 1, 0, small.data_ptr(),
                                       small.data_ptr(), small.data_ptr())
    assert st == bsort_gpu.BSORT_E_TOO_LARGE
