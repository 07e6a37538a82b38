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


def test_kernel_source_hash_ignores_comments_only():
    """A profile summary's counters stay attached to its kernel across edits
    of comments and layout, and are dropped once the code changes."""
    src = ('// header\n#include "x.cuh"\n/* block\n comment */ __global__ void k(float* p) {\n'
           '    p[0] = 1.0f;   // one\n    const char* s = "a // not a comment";\n    char c = \'/\';\n}\n')
    reworded = ('// another header, longer\n#include "x.cuh"\n__global__   void k(float* p)\n{\n'
                '    p[0] = 1.0f;\n    const char* s = "a // not a comment";  /* two */\n    char c = \'/\';\n}\n')
    changed = src.replace("1.0f", "2.0f")
    moved_string = src.replace('"a // not a comment"', '"a  // not a comment"')
    strip = bench.strip_comments
    assert strip(src) == strip(reworded).replace("k(float* p) {", "k(float* p) {")
    assert strip(src) != strip(changed)
    assert strip(src) != strip(moved_string)        # string literals are code, kept verbatim
    assert "block" not in strip(src) and "one" not in strip(src)
    assert '"a // not a comment"' in strip(src)
    for kernel in bench.KERNEL_FILE:
        assert len(bench.kernel_source_hash(kernel)) == 16
