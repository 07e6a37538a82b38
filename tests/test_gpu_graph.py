"""Device-driven solves (one CUDA graph per solve, conditional loops) and batches
of uneven solves in one graph launch: same results as the host-driven
solve_projection, and as the oracle within the parity tolerances."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S

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


def test_graph_solve_equals_host_loop(P):
    pb = tiny_problem()
    d = to_dev(pb)
    for prm in (P.default_params(pb["step"]), P.default_params(pb["step"], mu_min=0.0, max_iter=20, max_trials=30)):
        w_h, st_h = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
        sv = P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], prm)
        w_g, st_g = sv.solve(d["y"], np.zeros(3))
        assert np.array_equal(w_g, w_h), (w_g, w_h)
        assert st_g == st_h, (st_g, st_h)
        # the graph is reusable: a second launch from another start, another angle
        y2 = torch.from_numpy(O.drr_forward(O.warp_volume(pb["f0"], O.pca_dvf(None, pb["U"], pb["w_true"], pb["vol"]),
                                                          pb["vol"]), pb["vol"], dict(pb["cb"], angle=0.9),
                                            pb["step"]).astype(np.float32)).cuda()
        w3, st3 = sv.solve(y2, 0.5 * pb["w_true"], angle=0.9)
        w4, st4 = P.solve_projection(d["f0"], None, d["U"], y2, pb["vol"], dict(pb["cb"], angle=0.9),
                                     0.5 * pb["w_true"], prm)
        assert np.array_equal(w3, w4) and st3 == st4
        sv.close()


def test_graph_solve_matches_oracle_and_edge_cases(P):
    pb = tiny_problem()
    d = to_dev(pb)
    prm = P.default_params(pb["step"], mu_min=0.0, max_iter=20, max_trials=30)
    sv = P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], prm)
    w, st = sv.solve(d["y"], np.zeros(3))
    wo, sto, _ = O.solve_projection(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    assert np.linalg.norm(w - wo) < 2e-3 and st["J"] < st["J0"]
    with pytest.raises(P.PcasError) as e:                               # constant image
        sv.solve(torch.full_like(d["y"], 0.5), np.zeros(3))
    assert e.value.code == P.SINGULAR
    w2, st2 = sv.solve(d["y"], np.zeros(3))                             # still usable afterwards
    assert np.array_equal(w2, w)
    sv.close()
    sv0 = P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], P.default_params(pb["step"], max_iter=0))
    w0, st0 = sv0.solve(d["y"], np.full(3, 0.1))
    assert np.allclose(w0, 0.1) and st0["iters"] == 0 and st0["evals"] == 1
    sv0.close()


def test_batch_of_uneven_solves(P):
    """Six problems of different volumes, detectors, K and angles in one launch:
    each result equals its own single-solve graph (bitwise) and the host loop,
    and follows the oracle's solve (same iterations and evaluations, w within
    2e-3, tumour centroid within 0.05 mm)."""
    shapes = [((40, 36, 24, 4.0, 4.0, 4.0), 3, (64, 48, 4.0, 4.0)),
              ((61, 53, 29, 4.0, 3.5, 4.5), 5, (101, 77, 3.5, 3.5)),
              ((32, 32, 16, 4.0, 4.0, 4.0), 1, (48, 36, 4.0, 4.0)),
              ((48, 44, 20, 4.0, 4.0, 4.0), 3, (90, 60, 3.0, 3.0)),
              ((64, 64, 32, 4.0, 4.0, 4.0), 5, (128, 96, 3.1, 3.1)),
              ((36, 40, 28, 3.0, 3.0, 3.0), 2, (70, 50, 3.0, 3.0))]
    g = S.rng(50)
    probs, devs, solvers = [], [], []
    for i, (dims, K, det) in enumerate(shapes):
        ang = float(g.uniform(0, 2 * np.pi))
        w_true = g.standard_normal(K) * 0.5
        pb = make_problem(dims, K, det, ang, w_true, seeds=(60 + i, 70 + i, 80 + i))
        d = to_dev(pb)
        probs.append(pb)
        devs.append(d)
        solvers.append(P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], P.default_params(pb["step"])))
    batch = P.Batch(solvers, ys=[d["y"] for d in devs])
    angles = [pb["cb"]["angle"] for pb in probs]
    w_init = [np.zeros(pb["K"]) for pb in probs]
    ws, sts = batch.solve(angles, w_init)
    for i, (pb, d, sv) in enumerate(zip(probs, devs, solvers)):
        w1, st1 = sv.solve(d["y"], np.zeros(pb["K"]))
        assert np.array_equal(ws[i], w1) and sts[i] == st1, i
        wh, sth = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], np.zeros(pb["K"]),
                                     P.default_params(pb["step"]))
        assert np.array_equal(ws[i], wh), i
        wo, sto, _ = O.solve_projection(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], np.zeros(pb["K"]),
                                        P.default_params(pb["step"]))
        assert (sts[i]["iters"], sts[i]["evals"]) == (sto["iters"], sto["evals"]), (i, sts[i], sto)
        assert np.linalg.norm(ws[i] - wo) < 2e-3, (i, ws[i], wo)
        c, _ = P.localize_tumor(None, d["U"], ws[i], pb["vol"], pb["c_ref"])
        co, _ = O.localize_tumor(None, pb["U"], wo, pb["vol"], pb["c_ref"])
        assert np.linalg.norm(c - co) <= 0.05, (i, c, co)
    # relaunch with other starts: still consistent
    ws2, _ = batch.solve(angles, [0.3 * np.ones(pb["K"]) for pb in probs])
    w1, _ = solvers[0].solve(devs[0]["y"], 0.3 * np.ones(probs[0]["K"]))
    assert np.array_equal(ws2[0], w1)
    batch.close()
    for sv in solvers:
        sv.close()


def test_layout_follows_the_angle(P):
    """Views with |sin a| > |cos a| keep the solver volumes y-fastest.  One
    solver (x != y grid) walks through angles on both sides of every 45-degree
    boundary and back: each result equals the host-driven solve bitwise and the
    oracle's cost and gradient within the parity tolerances."""
    dims = (61, 47, 29, 4.0, 3.5, 4.5)
    w_true = np.array([0.6, -0.3, 0.4])
    pb = make_problem(dims, 3, (101, 77, 3.5, 3.5), 0.0, w_true, noise=0.0, seeds=(91, 92, 93))
    d = to_dev(pb)
    prm = P.default_params(pb["step"])
    sv = P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], prm)
    w_eval = 0.7 * w_true
    for ang in (0.3, 0.9, 2.0, 2.5, 3.3, 4.4, 5.0, 0.1, np.pi / 4 + 1e-3, np.pi / 4 - 1e-3):
        cb = dict(pb["cb"], angle=float(ang))
        y = O.drr_forward(O.warp_volume(pb["f0"], O.pca_dvf(None, pb["U"], w_true, pb["vol"]), pb["vol"]),
                          pb["vol"], cb, pb["step"]).astype(np.float32)
        yd = torch.from_numpy(y).cuda()
        w_g, st_g = sv.solve(yd, np.zeros(3), angle=ang)
        w_h, st_h = P.solve_projection(d["f0"], None, d["U"], yd, pb["vol"], cb, np.zeros(3), prm)
        assert np.array_equal(w_g, w_h) and st_g == st_h, ang
        J, G, _ = P.cost_grad(d["f0"], None, d["U"], w_eval, yd, pb["vol"], cb, pb["step"])
        Jo, Go, _ = O.cost_grad(pb["f0"], None, pb["U"], w_eval, y, pb["vol"], cb, pb["step"])
        assert abs(J - Jo) <= 1e-4 * Jo, (ang, J, Jo)
        assert np.linalg.norm(G - Go) <= 1e-3 * np.linalg.norm(Go), (ang, G, Go)
    sv.close()


@pytest.mark.parametrize("mu_min,max_trials", [(0.04, 30), (0.0, 7), (0.0, 6), (0.0, 1), (0.011, 4)])
def test_partial_batches_and_single_trials(P, mu_min, max_trials):
    """Schedules that fill a batch of five only partly (mu_min cuts it to 3 or
    4 steps, max_trials leaves 2 or 1, down to batches of one step): host loop
    and device-driven graph agree bitwise, and both follow the oracle's
    one-at-a-time rule."""
    pb = tiny_problem()
    d = to_dev(pb)
    prm = P.default_params(pb["step"], mu_min=mu_min, max_iter=12, max_trials=max_trials)
    w_h, st_h = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    sv = P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], prm)
    w_g, st_g = sv.solve(d["y"], np.zeros(3))
    sv.close()
    assert np.array_equal(w_g, w_h) and st_g == st_h
    wo, sto, _ = O.solve_projection(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    assert st_h["iters"] == sto["iters"] and st_h["evals"] == sto["evals"], (st_h, sto)
    assert np.linalg.norm(w_h - wo) < 2e-3, (w_h, wo)
