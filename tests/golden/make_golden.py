"""Writes tests/golden/digests.json: sha256 of the generated workloads and of
the oracle's (O2) output on the two paper-sized documents.

Calls only ``synth`` (the input generator) and ``oracle``; nothing here comes
from the CUDA path.  Re-run after a deliberate change to the generator:
    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def sha(b) -> str:
    return hashlib.sha256(bytes(b)).hexdigest()


def result_digest(res: dict) -> str:
    h = hashlib.sha256()
    h.update(np.asarray(res["counts"], dtype=np.uint64).tobytes())
    h.update(np.asarray(res["offsets"], dtype=np.uint32).tobytes())
    h.update(np.asarray(res["stream"], dtype=np.uint8).tobytes())
    return h.hexdigest()


def main() -> None:
    out = {"inputs": {}, "oracle_o2": {}, "batch_first16": []}
    for name in ("plain_190k", "plain_1m38", "plain_256m"):
        d = synth.plain(name)
        out["inputs"][name] = sha(d)
        if name != "plain_256m":
            r = oracle.stable(d, nthreads=8)
            out["oracle_o2"][name] = {"n_words": r["n_words"], "max_len": r["max_len"],
                                      "digest": result_digest(r)}
    for seed, n, v in synth.batch_shapes(16):
        out["batch_first16"].append({"seed": seed, "nbytes": n, "vocab": v,
                                     "sha256": sha(synth.batch_doc(seed, n, v))})
    with open(os.path.join(HERE, "digests.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
