"""Launch shapes (per size bucket) and the autotuner: every shape gives the
oracle's cost and gradient within the parity tolerances, device-driven and
host-driven solves agree bitwise under a tuned table, and the autotuner stores
a valid entry for the bucket."""
import numpy as np
import pytest

import oracle as O

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


@pytest.fixture(scope="module")
def prob():
    return make_problem((61, 53, 29, 4.0, 3.5, 4.5), 3, (101, 77, 3.5, 3.5), 1.1, np.array([0.7, -0.4, 0.3]),
                        seeds=(71, 72, 73))


SHAPES = [dict(ray_lw1=2, chunk1=0, voxel_tile=1, gather_per_sm=4, skip_empty=1, ray_lw4=[4] * 8, chunk=[12] * 8),
          dict(ray_lw1=4, chunk1=32, voxel_tile=2, gather_per_sm=16, skip_empty=0, ray_lw4=[2] * 8, chunk=[24] * 8),
          dict(ray_lw1=3, chunk1=64, voxel_tile=3, gather_per_sm=1, skip_empty=1, ray_lw4=[3] * 8, chunk=[16] * 8),
          dict(ray_lw1=2, chunk1=2, voxel_tile=4, gather_per_sm=26, skip_empty=1, ray_lw4=[2] * 8, chunk=[2] * 8),
          dict(ray_lw1=4, chunk1=128, voxel_tile=5, gather_per_sm=8, skip_empty=0, ray_lw4=[4] * 8, chunk=[64] * 8),
          dict(ray_lw1=3, chunk1=0, voxel_tile=0, gather_per_sm=8, skip_empty=1, ray_lw4=[2, 3, 4, 2, 3, 4, 2, 3],
               chunk=[12, 24, 16, 2, 64, 12, 16, 24])]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("swap", [0, 1])
def test_every_shape_matches_the_oracle(P, prob, shape, swap):
    pb = prob
    d = to_dev(pb)
    t = dict(shape, swap=[swap] * 8)
    P.tuning_set(pb["vol"], pb["cb"], 3, t)
    assert P.tuning_get(pb["vol"], pb["cb"], 3) == t
    w = np.array([0.4, -0.2, 0.1])
    J, G, _ = P.cost_grad(d["f0"], None, d["U"], w, d["y"], pb["vol"], pb["cb"], pb["step"])
    Jo, Go, _ = O.cost_grad(pb["f0"], None, pb["U"], w, pb["y"], pb["vol"], pb["cb"], pb["step"])
    assert abs(J - Jo) <= 1e-4 * Jo
    assert np.linalg.norm(G - Go) <= 1e-3 * np.linalg.norm(Go)
    prm = P.default_params(pb["step"])
    wh, sth = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    sv = P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], prm)
    wg, stg = sv.solve(d["y"], np.zeros(3))
    sv.close()
    assert np.array_equal(wg, wh) and stg == sth
    wo, _, _ = O.solve_projection(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    assert np.linalg.norm(wh - wo) < 2e-3
    P.tuning_clear()


def test_autotune_stores_a_valid_entry(P, prob):
    pb = prob
    d = to_dev(pb)
    P.tuning_clear()
    default = P.tuning_get(pb["vol"], pb["cb"], 3)
    assert default == dict(ray_lw1=3, chunk1=0, voxel_tile=0, gather_per_sm=8, skip_empty=1, ray_lw4=[3] * 8,
                           chunk=[16] * 8, swap=[0, 0, 0, 1, 1, 1, 0, 0])
    prm = P.default_params(pb["step"])
    t = P.autotune(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], prm)
    print("autotuned:", t)
    assert t == P.tuning_get(pb["vol"], pb["cb"], 3)
    assert 2 <= t["ray_lw1"] <= 4 and t["chunk1"] in (0, 32, 64)
    assert all(2 <= v <= 4 for v in t["ray_lw4"]) and all(v in (12, 16, 24) for v in t["chunk"])
    assert 0 <= t["voxel_tile"] < 6 and t["gather_per_sm"] in (4, 8, 16) and t["skip_empty"] in (0, 1)
    # the tuned table drives both solve paths identically, within parity of the oracle
    wh, sth = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    sv = P.Solver(d["f0"], None, d["U"], pb["vol"], pb["cb"], prm)
    wg, stg = sv.solve(d["y"], np.zeros(3))
    sv.close()
    assert np.array_equal(wg, wh) and stg == sth
    wo, _, _ = O.solve_projection(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    assert np.linalg.norm(wh - wo) < 2e-3
    # another bucket is untouched; clearing restores the defaults
    other = dict(pb["cb"], nu=301)
    assert P.tuning_get(pb["vol"], other, 3) == default
    P.tuning_clear()
    assert P.tuning_get(pb["vol"], pb["cb"], 3) == default
