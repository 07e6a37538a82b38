"""Writes tests/golden/bench_truth.json: the tumour centroid at the planted
coefficients of every projection of the benchmark workloads, found by the
FP64 oracle's localisation (Sec. II.A: the fixed point y <- -x(c_ref + y) of
the pull-back DVF, tolerance 1e-6 mm, at most 50 iterations).  These are the
truth of the benchmark's mm error.  Each entry carries a fingerprint of the
inputs it belongs to (bench.input_fingerprint), so that a changed input recipe
is noticed instead of measured against stale values.

Inputs come from the benchmark's own recipes (bench.make_inputs,
bench.precision_inputs, bench.batch_inputs: seeded generators, no arithmetic
of the method); every value written comes from the oracle.

    python tests/golden/make_bench_truth.py          # about a minute, ~12 GB of host memory
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import bench  # noqa: E402  (input recipes only)
import oracle as O  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "bench_truth.json")


def centroids(U, trace, vol, c_ref):
    U64 = np.ascontiguousarray(U, dtype=np.float64)         # converted once, reused by every call
    out = []
    for w in trace:
        c, ok = O.localize_tumor(None, U64, w, vol, c_ref)
        out.append([round(float(v), 7) for v in c])
    return out


def main():
    O.build()
    rec = {"generator": "tests/golden/make_bench_truth.py",
           "what": "tumour centroid (mm) at the planted coefficients, FP64 oracle localisation (Sec. II.A), "
                   "50 iterations at most, tolerance 1e-6 mm"}
    for name, irregular in (("sequence-regular", False), ("sequence-irregular", True)):
        vol, f0, c_ref, U, trace, train, angles = bench.make_inputs(irregular)
        rec[name] = {"fingerprint": bench.input_fingerprint(trace, c_ref, U),
                     "c_true": centroids(U, trace, vol, c_ref)}
        print(name, len(trace), flush=True)
    vol, f0, c_ref, U, trace, train, angles = bench.precision_inputs()
    rec["precision"] = {"fingerprint": bench.input_fingerprint(trace, c_ref, U),
                        "c_true": centroids(U, trace, vol, c_ref)}
    print("precision", len(trace), flush=True)
    del U, f0
    probs = bench.batch_inputs()
    c_b = []
    for pb in probs:
        c_b += centroids(pb["U"], [pb["w_true"]], pb["vol"], pb["c_ref"])
    rec["batch"] = {"fingerprint": bench.input_fingerprint(*bench.batch_fingerprint_parts(probs)), "c_true": c_b}
    print("batch", len(c_b), flush=True)
    with open(OUT, "w") as fh:
        json.dump(rec, fh, separators=(",", ":"))
        fh.write("\n")


if __name__ == "__main__":
    main()
