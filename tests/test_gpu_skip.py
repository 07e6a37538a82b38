"""Empty-space skipping of the solver projectors (occupancy bricks of 4^3
voxels marked by the warp kernels): exact by construction, so every result
with skipping on equals the result with it off bit for bit -- costs and
gradients, host-driven and device-driven solves, both volume layouts, rays
that miss the object, and rays whose walk through empty bricks runs out of
steps -- and stays within the parity tolerances of the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S

from cases import make_problem, to_dev

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
    yield pcasolve
    pcasolve.tuning_clear()


def _set_skip(P, vol, cb, K, skip):
    t = P.tuning_get(vol, cb, K)
    t["skip_empty"] = skip
    P.tuning_set(vol, cb, K, t)


def _both(P, vol, cb, K, fn):
    out = []
    for skip in (0, 1):
        _set_skip(P, vol, cb, K, skip)
        out.append(fn())
    P.tuning_clear()
    return out


@pytest.mark.parametrize("angle", [0.0, 0.7, 1.5, 2.4, 3.9])
def test_solves_equal_with_and_without_skipping(P, angle):
    """The angles cover both layouts (y fastest in the bins around 90 deg)."""
    pb = make_problem((61, 53, 29, 4.0, 3.5, 4.5), 3, (101, 77, 3.5, 3.5), angle, np.array([0.7, -0.4, 0.3]),
                      seeds=(81, 82, 83))
    d = to_dev(pb)
    prm = P.default_params(pb["step"])
    w_eval = np.array([0.4, -0.2, 0.1])

    def run():
        J, G, ab = P.cost_grad(d["f0"], None, d["U"], w_eval, d["y"], pb["vol"], pb["cb"], pb["step"])
        wh, sth = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
        sv = P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], prm)
        wg, stg = sv.solve(d["y"], np.zeros(3))
        sv.close()
        return J, G, ab, wh, sth, wg, stg

    off, on = _both(P, pb["vol"], pb["cb"], 3, run)
    J0, G0, ab0, wh0, st0, wg0, sg0 = off
    J1, G1, ab1, wh1, st1, wg1, sg1 = on
    assert J0 == J1 and np.array_equal(G0, G1) and np.array_equal(ab0, ab1)
    assert np.array_equal(wh0, wh1) and st0 == st1
    assert np.array_equal(wg1, wh1) and sg1 == st1 and np.array_equal(wg0, wg1)
    Jo, Go, _ = O.cost_grad(pb["f0"], None, pb["U"], w_eval, pb["y"], pb["vol"], pb["cb"], pb["step"])
    assert abs(J1 - Jo) <= 1e-4 * Jo
    assert np.linalg.norm(G1 - Go) <= 1e-3 * np.linalg.norm(Go)


def _long_problem():
    """A 400-voxel-long box of air with a small object at its far end (from a
    source at +x) and one off to the side: rays at 90 deg cross about a hundred
    empty bricks before the object, more than a walk takes, and many rays
    miss the object entirely."""
    vol = S.volume(400, 24, 16, 1.0, 1.0, 1.0)
    f0 = np.zeros((16, 24, 400), np.float32)
    g = S.rng(5)
    f0[4:12, 6:18, 3:11] = 0.02 + 0.01 * g.random((8, 12, 8), dtype=np.float32)
    f0[5:9, 2:6, 200:206] = 0.015
    K = 2
    U = S.eigen_dvfs(vol, K, seed=6)
    cb = S.cone_beam(96, 40, 1.2, 1.2, np.pi / 2)
    step = 0.5
    w_true = np.array([0.5, -0.3])
    y = O.drr_forward(O.warp_volume(f0, O.pca_dvf(None, U, w_true, vol), vol), vol, cb, step).astype(np.float32)
    return vol, cb, step, f0, U, y


def test_long_walks_and_missed_rays(P):
    vol, cb, step, f0, U, y = _long_problem()
    tf0, tU, ty = (torch.from_numpy(a.ravel()).cuda() for a in (f0, U, y))
    ty = ty.view(y.shape)
    w = np.array([0.3, -0.2])
    for ang in (np.pi / 2, np.pi / 2 + 0.2, 0.05):
        c = dict(cb, angle=float(ang))
        yo = O.drr_forward(O.warp_volume(f0, O.pca_dvf(None, U, np.array([0.5, -0.3]), vol), vol), vol, c,
                           step).astype(np.float32)
        tyo = torch.from_numpy(yo).cuda()
        off, on = _both(P, vol, c, 2, lambda: P.cost_grad(tf0, None, tU, w, tyo, vol, c, step))
        assert off[0] == on[0] and np.array_equal(off[1], on[1]), ang
        Jo, Go, _ = O.cost_grad(f0, None, U, w, yo, vol, c, step)
        assert abs(on[0] - Jo) <= 1e-4 * Jo, (ang, on[0], Jo)
        assert np.linalg.norm(on[1] - Go) <= 1e-3 * np.linalg.norm(Go), ang
    prm = P.default_params(step)
    off, on = _both(P, vol, cb, 2,
                    lambda: P.solve_projection(tf0, None, tU, ty, vol, cb, np.zeros(2), prm))
    assert np.array_equal(off[0], on[0]) and off[1] == on[1]
