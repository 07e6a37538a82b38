"""cost_grad_static: the cost/gradient evaluation for callers that cannot
allocate device memory (allocation-free real-time loops, or a host program
that owns all device memory).  It must give what cost_grad gives with a
caller workspace, call after call, although its fixed device scratch keeps
the previous call's contents.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import oracle as O

from cases import make_problem, tiny_problem, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1102_1712_gb300 import build as B
    B.build()
    from paper_1102_1712_gb300 import pcasolve
    pcasolve.lib()
    return pcasolve


def _close(a, b):
    (J, G, (x, y)), (Jr, Gr, (xr, yr)) = a, b
    assert abs(J - Jr) <= 1e-4 * abs(Jr)
    assert np.linalg.norm(G - Gr) <= 1e-3 * np.linalg.norm(Gr)
    assert abs(x - xr) <= 1e-5 * abs(xr) and abs(y - yr) <= 1e-5 * max(abs(xr), abs(yr))


def test_static_scratch_matches_workspace_call_twice(P):
    pb = tiny_problem()
    d = to_dev(pb)
    args = (pb["vol"], pb["cb"], pb["step"])
    for w in (np.array([0.5, 0.5, -0.5]), np.array([-0.8, 0.2, 0.9])):     # two calls in a row
        got = P.cost_grad_static(d["f0"], None, d["U"], w, d["y"], *args)
        ref = P.cost_grad(d["f0"], None, d["U"], w, d["y"], *args)
        _close(got, ref)
    # a different, smaller problem right after: stale contents must not leak in
    pb2 = make_problem((40, 36, 24, 4.0, 4.0, 4.0), 1, (64, 48, 4.0, 4.0), 1.9, (0.6,), seeds=(21, 22, 23))
    d2 = to_dev(pb2)
    w = np.array([0.3])
    got = P.cost_grad_static(d2["f0"], None, d2["U"], w, d2["y"], pb2["vol"], pb2["cb"], pb2["step"])
    ref = P.cost_grad(d2["f0"], None, d2["U"], w, d2["y"], pb2["vol"], pb2["cb"], pb2["step"])
    _close(got, ref)
    # and it still agrees with the FP64 oracle
    Jo, Go, _ = O.cost_grad(pb2["f0"], None, pb2["U"], w, pb2["y"], pb2["vol"], pb2["cb"], pb2["step"])
    assert abs(got[0] - Jo) <= 1e-4 * Jo and np.linalg.norm(got[1] - Go) <= 1e-3 * np.linalg.norm(Go)


def test_static_scratch_rejects_oversized_problems(P):
    from paper_1102_1712_gb300 import synth as S
    vol = S.volume(256, 256, 100, 2.0, 2.0, 2.5)
    cb = S.cone_beam(512, 384, 0.776, 0.776)
    assert P.workspace_bytes(vol, cb, 3) > 16 * 1024 * 1024
    N = 256 * 256 * 100
    f0 = torch.zeros(N, device="cuda")
    U = torch.zeros(3 * 3 * N, device="cuda")
    y = torch.zeros(512 * 384, device="cuda")
    with pytest.raises(P.PcasError) as e:
        P.cost_grad_static(f0, None, U, np.zeros(3), y, vol, cb, 1.0)
    assert e.value.code == P.INVALID_ARG and "static scratch" in str(e.value)
