"""drr_siddon (Siddon's exact radiological path, Sec. II.B's simulation
projector) against the oracle's Siddon, and solves on Siddon-rendered images
(no inverse crime: the measured image is not made by the solver's projector)."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S

from cases import SEQUENCE, TINY, make_problem

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


CASES = [((64, 64, 32, 4.0, 4.0, 4.0), (128, 96, 3.1, 3.1), 0.0, (0.0, 0.0)),
         ((61, 53, 29, 4.0, 3.5, 4.5), (101, 77, 3.5, 3.5), 2.2, (3.0, -2.0)),
         ((40, 36, 24, 4.0, 4.0, 4.0), (64, 49, 4.0, 4.0), np.pi / 2, (0.0, 0.0)),
         ((33, 47, 21, 3.0, 3.0, 5.0), (90, 60, 3.0, 3.0), 4.0, (-5.0, 7.0))]


@pytest.mark.parametrize("dims,det,angle,off", CASES)
def test_siddon_matches_oracle(P, dims, det, angle, off):
    vol = S.volume(*dims)
    f0, _ = S.phantom(vol, 12.0, seed=41)
    f = f0 + S.gaussian_noise(f0.shape, 0.002, seed=42)          # not piecewise flat
    cb = S.cone_beam(det[0], det[1], det[2], det[3], angle, off_u=off[0], off_v=off[1])
    p = P.drr_siddon(torch.from_numpy(f.ravel()).cuda(), vol, cb).cpu().numpy().astype(np.float64)
    po = O.siddon_forward(f.astype(np.float64), vol, cb)
    err = np.abs(p - po).max()
    print(f"siddon {dims} angle {angle:.2f}: max |d| = {err:.2e} of max {np.abs(po).max():.3f}")
    assert err <= 1e-6 * np.abs(po).max()


def test_siddon_sequence_size_sampled(P):
    s = SEQUENCE
    vol = S.volume(*s["vol"])
    f0, _ = S.phantom(vol, s["tumor"], seed=s["seeds"][0])
    cb = S.cone_beam(*s["det"], 1.234)
    p = P.drr_siddon(torch.from_numpy(f0.ravel()).cuda(), vol, cb).cpu().numpy()
    g = S.rng(43)
    iu, iv = g.integers(0, cb["nu"], 200), g.integers(0, cb["nv"], 200)
    ref = np.array([O.siddon_ray(f0, vol, cb, a, b) for a, b in zip(iu, iv)])
    got = p.reshape(cb["nv"], cb["nu"])[iv, iu].astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-6 * max(np.abs(ref).max(), 1.0)


def test_siddon_rejects_bad_input(P):
    vol = S.volume(16, 16, 8, 2.0, 2.0, 2.0)
    f = torch.zeros(16 * 16 * 8, device="cuda")
    with pytest.raises(P.PcasError):
        P.drr_siddon(f, vol, S.cone_beam(8, 8, 1.0, 1.0, 0.0, sad=5.0))        # source inside the volume
    with pytest.raises((P.PcasError, ValueError)):                            # binding or library check
        P.drr_siddon(f, dict(vol, nx=0), S.cone_beam(8, 8, 1.0, 1.0))


def test_solve_on_siddon_rendered_image(P):
    """The tiny workload with the measured image rendered by Siddon's projector
    (voxel cubes, exact chords) instead of the solver's trilinear march: the
    GPU and the oracle agree on the solve, and the planted w is recovered up
    to the projector mismatch."""
    t = TINY
    pb = make_problem(t["vol"], t["K"], t["det"], t["angle"], t["w_true"], noise=0.0, seeds=t["seeds"],
                      tumor=t["tumor"])
    vol, cb = pb["vol"], pb["cb"]
    f_true = O.warp_volume(pb["f0"], O.pca_dvf(None, pb["U"], pb["w_true"], vol), vol)
    y = O.siddon_forward(f_true, vol, cb)
    y = (y + S.gaussian_noise(y.shape, t["noise"] * np.abs(y).max(), seed=t["seeds"][2], dtype=np.float64))
    y = y.astype(np.float32)
    prm = P.default_params(pb["step"], mu_min=0.0, max_iter=t["iters"], max_trials=30)
    d = {k: torch.from_numpy(pb[k].ravel()).cuda() for k in ("f0", "U")}
    w, st = P.solve_projection(d["f0"], None, d["U"], torch.from_numpy(y).cuda(), vol, cb, np.zeros(3), prm)
    wo, sto, _ = O.solve_projection(pb["f0"], None, pb["U"], y, vol, cb, np.zeros(3), prm)
    print(f"siddon-rendered tiny solve: w = {w}, oracle {wo}, planted {pb['w_true']}")
    assert np.linalg.norm(w - wo) < 2e-3
    assert np.linalg.norm(w - pb["w_true"]) < 0.1 * np.linalg.norm(pb["w_true"])
    c, _ = P.localize_tumor(None, d["U"], w, vol, pb["c_ref"])
    ct, _ = O.localize_tumor(None, pb["U"], pb["w_true"], vol, pb["c_ref"])
    assert np.linalg.norm(c - ct) < 1.0
