"""The stored truth of the benchmark's mm error (tests/golden/bench_truth.json)
belongs to the benchmark's current input recipes and is the oracle's
localisation at the planted coefficients (Sec. II.A)."""
import os
import sys

import numpy as np

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_sequence_truth_is_the_oracle_localisation():
    for name, irregular in (("sequence-regular", False), ("sequence-irregular", True)):
        vol, f0, c_ref, U, trace, train, angles = bench.make_inputs(irregular)
        c_true = bench.truth(name, trace, c_ref, U)         # raises on other inputs
        assert c_true.shape == (len(trace), 3)
        U64 = U.astype(np.float64)
        for t in (0, 17, 311, len(trace) - 1):
            c, ok = O.localize_tumor(None, U64, trace[t], vol, c_ref)
            assert np.abs(c - c_true[t]).max() <= 1e-6, (name, t)


def test_batch_truth_is_the_oracle_localisation():
    probs = bench.batch_inputs()
    c_true = bench.truth("batch", *bench.batch_fingerprint_parts(probs))
    assert c_true.shape == (len(probs), 3)
    for i in (0, 5, 63):
        pb = probs[i]
        c, _ = O.localize_tumor(None, pb["U"], pb["w_true"], pb["vol"], pb["c_ref"])
        assert np.abs(c - c_true[i]).max() <= 1e-6, i


def test_changed_inputs_are_refused():
    vol, f0, c_ref, U, trace, train, angles = bench.make_inputs(False)
    try:
        bench.truth("sequence-regular", trace * (1 + 1e-3), c_ref, U)
    except SystemExit:
        return
    raise AssertionError("a changed trace was accepted")
