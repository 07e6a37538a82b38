"""Runs of consecutive projections on a device-driven solver: the Eq. (3)
warm start and the Sec. II.A localisation inside the graph give bitwise the
results of the per-projection loop (solve + host lp_predict + host
localize_tumor), for device and pinned-host images, across layout flips,
past the 64-slot ring, and when a run is resumed from a given history; a
constant image in the middle of a run is reported and the run goes on."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S

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


@pytest.fixture(scope="module")
def seq():
    """A short breathing sequence on the tiny volume, images rendered by the
    oracle's Siddon projector at angles that sweep through every layout bin."""
    vol = S.volume(64, 64, 32, 4.0, 4.0, 4.0)
    f0, c_ref = S.phantom(vol, 15.0, seed=31)
    K = 3
    U = S.eigen_dvfs(vol, K, seed=32)
    n = 12
    trace = S.breathing_trace(n, 10.0, 4.0, 12.0, K=K, seed=33)
    train = S.breathing_trace(200, 10.0, 4.0, 12.0, K=K, t0=0.37)
    angles = np.linspace(0.0, 2.6, n)
    cb = S.cone_beam(128, 96, 3.1, 3.1, 0.0)
    ys = []
    for t in range(n):
        f = O.warp_volume(f0, O.pca_dvf(None, U, trace[t], vol), vol)
        ys.append(O.siddon_forward(f, vol, dict(cb, angle=float(angles[t]))).astype(np.float32))
    return dict(vol=vol, f0=f0, c_ref=c_ref, U=U, K=K, trace=trace, c_lp=O.lp_fit(train, 2), angles=angles,
                cb=cb, ys=ys, step=2.0)


def _loop(P, sv, d, ys_dev, t0, t1, hist):
    """The per-projection reference: graph solve, host warm start, host localisation."""
    out = []
    for t in range(t0, t1):
        if not hist:
            w0 = np.zeros(d["K"])
        elif len(hist) < 2:
            w0 = hist[-1]
        else:
            w0 = P.lp_predict(np.stack([hist[-1], hist[-2]]), d["c_lp"])
        w, st = sv.solve(ys_dev[t], w0, angle=float(d["angles"][t]))
        c, conv = P.localize_tumor(None, d["tU"], w, d["vol"], d["c_ref"])
        hist.append(w)
        out.append((w, st, c, conv))
    return out


def _same(a, b):
    for (w1, s1, c1, k1), (w2, s2, c2, k2) in zip(a, b):
        assert np.array_equal(w1, w2) and s1 == s2 and np.array_equal(c1, c2) and k1 == k2


def test_run_equals_the_projection_loop(P, seq):
    d = dict(seq)
    dev = "cuda"
    d["tU"] = torch.from_numpy(seq["U"].ravel()).to(dev)
    tf0 = torch.from_numpy(seq["f0"].ravel()).to(dev)
    ys_dev = [torch.from_numpy(y.ravel()).to(dev) for y in seq["ys"]]
    prm = P.default_params(seq["step"])
    n = len(seq["ys"])
    ref = _loop(P, P.Solver(tf0, None, d["tU"], seq["vol"], seq["cb"], prm), d, ys_dev, 0, n, [])
    sv = P.Solver(tf0, None, d["tU"], seq["vol"], seq["cb"], prm)
    sv.seq_begin(seq["c_lp"], seq["c_ref"])
    got = sv.solve_sequence(ys_dev, seq["angles"], w_first=np.zeros(seq["K"]), lookahead=5)
    _same(got, ref)
    # resumed from a given history: the second half as its own run
    h = n // 2
    sv.seq_begin(seq["c_lp"], seq["c_ref"], w_hist=[ref[h - 1][0], ref[h - 2][0]])
    _same(sv.solve_sequence(ys_dev[h:], seq["angles"][h:]), ref[h:])
    # pinned host images (copied inside each queued solve)
    ys_host = [torch.from_numpy(y.ravel()).pin_memory() for y in seq["ys"]]
    sv.seq_begin(seq["c_lp"], seq["c_ref"])
    _same(sv.solve_sequence(ys_host, seq["angles"], w_first=np.zeros(seq["K"])), ref)
    # the solutions track the planted trace and the centroids their truth
    for t, (w, st, c, conv) in enumerate(got):
        ct, _ = P.localize_tumor(None, d["tU"], seq["trace"][t], seq["vol"], seq["c_ref"])
        assert conv and np.linalg.norm(c - ct) < 1.0, (t, c, ct)
    sv.close()


def test_long_run_wraps_the_ring_and_errors(P, seq):
    d = dict(seq)
    d["tU"] = torch.from_numpy(seq["U"].ravel()).cuda()
    tf0 = torch.from_numpy(seq["f0"].ravel()).cuda()
    prm = P.default_params(seq["step"], max_iter=2)
    n = 70                                   # more than the 64 slots of the ring
    idx = [t % len(seq["ys"]) for t in range(n)]
    ys_dev = [torch.from_numpy(seq["ys"][i].ravel()).cuda() for i in idx]
    d["angles"] = np.array([seq["angles"][i] for i in idx])
    ref = _loop(P, P.Solver(tf0, None, d["tU"], seq["vol"], seq["cb"], prm), d, ys_dev, 0, n, [])
    sv = P.Solver(tf0, None, d["tU"], seq["vol"], seq["cb"], prm)
    with pytest.raises(P.PcasError):                       # no run begun
        sv.seq_enqueue(ys_dev[0], 0.0)
    sv.seq_begin(seq["c_lp"], seq["c_ref"])
    _same(sv.solve_sequence(ys_dev, d["angles"], lookahead=40), ref)
    with pytest.raises(P.PcasError):                       # long gone from the ring
        sv.seq_result(0)
    # a constant image mid-run: reported, and the run continues from its start
    sv.seq_begin(seq["c_lp"], seq["c_ref"])
    t0 = sv.seq_enqueue(ys_dev[0], float(d["angles"][0]))
    t1 = sv.seq_enqueue(torch.full_like(ys_dev[1], 0.5), float(d["angles"][1]))
    t2 = sv.seq_enqueue(ys_dev[2], float(d["angles"][2]))
    w0, _, _, _ = sv.seq_result(t0)
    with pytest.raises(P.PcasError) as e:
        sv.seq_result(t1)
    assert e.value.code == P.SINGULAR
    w2, st2, _, _ = sv.seq_result(t2)
    assert np.all(np.isfinite(w2)) and st2["status"] == P.OK
    sv.close()
