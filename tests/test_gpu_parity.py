"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded
inputs, element by element where the oracle can afford it.

Tolerances (float32 GPU path against float64 oracle):
  DRR            max |dp| <= 1e-4 * max |p_oracle|        (stated target)
  dJ/dw          ||dG|| <= 1e-3 * ||G_oracle||              (stated target)
  tumour centroid |dc| <= 0.05 mm                            (stated target)
  DVF            max |d| <= 2e-6 * max |dvf|  (K+1 FP32 FMAs of O(10 mm) terms)
  warp           max |df| <= 5e-5 * max |f0|  (FP32 position i + x/s carries
                 up to ~1.5e-5 voxel of rounding for i < 256, times a jump of
                 at most max|f0| per voxel, plus margin)
  P^T            max |dg| <= 1e-4 * max |g_oracle| (same rounding allowance as P)
  J, (a, b)      relative 1e-4 / 1e-5 (FP32 sums of positive terms; FP64 across blocks)
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S

from cases import SEQUENCE, TINY, make_problem, tiny_problem, to_dev

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
def tiny():
    return tiny_problem()


def np32(t):
    return t.detach().cpu().numpy().astype(np.float64)


# ------------------------------------------------------------------ Eq. (1)
@pytest.mark.parametrize("dims,K,with_mean", [((64, 64, 32, 4.0, 4.0, 4.0), 3, False),
                                               ((61, 53, 29, 4.0, 3.5, 4.5), 5, True),
                                               ((8, 8, 1, 4.0, 4.0, 4.0), 1, True)])
def test_pca_dvf(P, dims, K, with_mean):
    vol = S.volume(*dims)
    U = S.eigen_dvfs(vol, K, seed=4)
    mean = (0.5 * U[0]).copy() if with_mean else None
    w = np.linspace(-1.1, 0.9, K)
    tU = torch.from_numpy(U.ravel()).cuda()
    tm = None if mean is None else torch.from_numpy(mean.ravel()).cuda()
    got = np32(P.pca_dvf(tm, tU, w, vol))
    ref = O.pca_dvf(mean, U, w, vol).ravel()
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


# ------------------------------------------------------------ Eq. (A.3/A.5)
@pytest.mark.parametrize("dims", [(64, 64, 32, 4.0, 4.0, 4.0), (61, 53, 29, 4.0, 3.5, 4.5),
                                  (7, 5, 1, 2.0, 2.0, 2.0)])
def test_warp_volume(P, dims):
    vol = S.volume(*dims)
    f0, _ = S.phantom(vol, 10.0, seed=5)
    f0 = f0 + S.rng(6).uniform(0, 0.01, f0.shape).astype(np.float32)      # no flat regions
    U = S.eigen_dvfs(vol, 2, seed=7)
    dvf = (1.7 * U[0] - 0.8 * U[1]).astype(np.float32)                    # up to ~25 mm
    got = np32(P.warp_volume(torch.from_numpy(f0.ravel()).cuda(), torch.from_numpy(dvf.ravel()).cuda(), vol))
    ref = O.warp_volume(f0, dvf, vol)
    assert np.abs(got - ref).max() <= 5e-5 * np.abs(f0).max()
    # identity warp is exact
    z = torch.zeros(3 * f0.size, device="cuda")
    assert np.array_equal(np32(P.warp_volume(torch.from_numpy(f0.ravel()).cuda(), z, vol)), f0.ravel())


# --------------------------------------------------------------- P (Eq. 2)
DRR_CASES = [
    ((64, 64, 32, 4.0, 4.0, 4.0), (128, 96, 3.1, 3.1), 0.0, (0.0, 0.0)),
    ((64, 64, 32, 4.0, 4.0, 4.0), (127, 95, 3.1, 3.3), 2.3, (7.0, -5.0)),   # ragged tiles
    ((61, 53, 29, 4.0, 3.5, 4.5), (100, 70, 4.0, 4.0), 0.9, (0.0, 0.0)),
    ((40, 40, 1, 4.0, 4.0, 4.0), (64, 9, 3.0, 3.0), 1.2, (0.0, 0.0)),        # one-voxel-thick volume
    ((32, 32, 16, 4.0, 4.0, 4.0), (1, 1, 3.0, 3.0), 0.4, (0.0, 0.0)),        # single pixel
]


@pytest.mark.parametrize("dims,det,angle,off", DRR_CASES)
def test_drr_forward(P, dims, det, angle, off):
    vol = S.volume(*dims)
    f0, _ = S.phantom(vol, 10.0, seed=8)
    cb = S.cone_beam(det[0], det[1], det[2], det[3], angle, off_u=off[0], off_v=off[1])
    step = 0.5 * min(dims[3:])
    got = np32(P.drr_forward(torch.from_numpy(f0.ravel()).cuda(), vol, cb, step))
    ref = O.drr_forward(f0, vol, cb, step)
    scale = max(np.abs(ref).max(), 1e-30)
    assert np.abs(got - ref).max() <= 1e-4 * scale


def test_drr_rays_missing_volume_are_zero(P):
    vol = S.volume(32, 32, 16, 4.0, 4.0, 4.0)
    f = torch.ones(32 * 32 * 16, device="cuda")
    cb = S.cone_beam(16, 16, 2.0, 2.0, 0.5, off_u=900.0)
    assert torch.count_nonzero(P.drr_forward(f, vol, cb, 2.0)).item() == 0


# --------------------------------------------------------------------- P^T
@pytest.mark.parametrize("dims,det,angle,off", DRR_CASES[:4])
def test_drr_adjoint(P, dims, det, angle, off):
    vol = S.volume(*dims)
    cb = S.cone_beam(det[0], det[1], det[2], det[3], angle, off_u=off[0], off_v=off[1])
    step = 0.5 * min(dims[3:])
    img = S.rng(9).uniform(-1, 1, det[0] * det[1]).astype(np.float32)
    got = np32(P.drr_adjoint(torch.from_numpy(img).cuda(), vol, cb, step))
    ref = O.drr_adjoint(img, vol, cb, step)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


def test_gpu_adjoint_identity(P):
    """<P x, y> = <x, P^T y> for the GPU pair itself (float32 rounding only)."""
    vol = S.volume(48, 44, 20, 4.0, 4.0, 4.0)
    cb = S.cone_beam(90, 60, 3.0, 3.0, 0.8, off_u=4.0)
    g = S.rng(10)
    x = torch.from_numpy(g.uniform(0, 1, 48 * 44 * 20).astype(np.float32)).cuda()
    y = torch.from_numpy(g.uniform(0, 1, 90 * 60).astype(np.float32)).cuda()
    lhs = float((P.drr_forward(x, vol, cb, 2.0).double() * y.double()).sum())
    rhs = float((x.double() * P.drr_adjoint(y, vol, cb, 2.0).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


# ------------------------------------------------- cost and gradient (A.1, A.2)
@pytest.mark.parametrize("w", [(0.0, 0.0, 0.0), (1.2, -0.4, 0.3), (0.5, 0.5, -0.5), (-0.8, 0.2, 0.9)])
def test_cost_grad_tiny(P, tiny, w):
    d = to_dev(tiny)
    w = np.asarray(w, float)
    J, G, (a, b) = P.cost_grad(d["f0"], d["mean"], d["U"], w, d["y"], tiny["vol"], tiny["cb"], tiny["step"])
    Jo, Go, (ao, bo) = O.cost_grad(tiny["f0"], None, tiny["U"], w, tiny["y"], tiny["vol"], tiny["cb"], tiny["step"])
    assert abs(J - Jo) <= 1e-4 * Jo
    assert abs(a - ao) <= 1e-5 * abs(ao) and abs(b - bo) <= 1e-5 * max(abs(ao), abs(bo))
    if np.linalg.norm(w - tiny["w_true"]) > 0.1:     # away from the optimum where G -> 0
        assert np.linalg.norm(G - Go) <= 1e-3 * np.linalg.norm(Go), (G, Go)


@pytest.mark.parametrize("K,with_mean,dims,det,angle", [
    (1, False, (40, 36, 24, 4.0, 4.0, 4.0), (64, 48, 4.0, 4.0), 1.9),
    (5, True, (61, 53, 29, 4.0, 3.5, 4.5), (101, 77, 3.5, 3.5), 4.0),
])
def test_cost_grad_variants(P, K, with_mean, dims, det, angle):
    w_true = np.linspace(0.6, -0.4, K)
    pb = make_problem(dims, K, det, angle, w_true, with_mean=with_mean, seeds=(21, 22, 23))
    d = to_dev(pb)
    w = 0.3 * np.ones(K)
    J, G, ab = P.cost_grad(d["f0"], d["mean"], d["U"], w, d["y"], pb["vol"], pb["cb"], pb["step"])
    Jo, Go, abo = O.cost_grad(pb["f0"], pb["mean"], pb["U"], w, pb["y"], pb["vol"], pb["cb"], pb["step"])
    assert abs(J - Jo) <= 1e-4 * Jo
    assert np.linalg.norm(G - Go) <= 1e-3 * np.linalg.norm(Go), (G, Go)


def test_cost_grad_singular_image(P, tiny):
    d = to_dev(tiny)
    y = torch.full_like(d["y"], 0.25)
    with pytest.raises(P.PcasError) as e:
        P.cost_grad(d["f0"], None, d["U"], np.zeros(3), y, tiny["vol"], tiny["cb"], tiny["step"])
    assert e.value.code == P.SINGULAR


# ---------------------------------------------------------- the full solve
def test_solve_tiny_matches_oracle(P, tiny):
    """Tiny workload: 20 iterations from w = 0, backtracking down to tiny steps."""
    d = to_dev(tiny)
    prm = P.default_params(tiny["step"], mu_min=0.0, max_iter=TINY["iters"], max_trials=30)
    w, st = P.solve_projection(d["f0"], d["mean"], d["U"], d["y"], tiny["vol"], tiny["cb"], np.zeros(3), prm)
    wo, sto, trace = O.solve_projection(tiny["f0"], None, tiny["U"], tiny["y"], tiny["vol"], tiny["cb"],
                                        np.zeros(3), prm)
    assert st["J"] < st["J0"] and abs(st["J0"] - sto["J0"]) <= 1e-4 * sto["J0"]
    assert np.all(np.diff(trace) <= 1e-12 * trace[0])       # monotone up to FP64 rounding
    assert np.linalg.norm(w - wo) < 2e-3, (w, wo, st, sto)
    c, ok = P.localize_tumor(None, d["U"], w, tiny["vol"], tiny["c_ref"])
    co, oko = O.localize_tumor(None, tiny["U"], wo, tiny["vol"], tiny["c_ref"])
    assert ok and oko and np.abs(c - co).max() <= 0.05
    ct, _ = O.localize_tumor(None, tiny["U"], tiny["w_true"], tiny["vol"], tiny["c_ref"])
    assert np.linalg.norm(c - ct) < 1.0       # 1 % noise: sub-mm localisation


def test_solve_paper_rule_stops_and_counts(P, tiny):
    """Appendix rules with scaled constants: stop when no mu >= mu_min passes; the
    GPU and oracle agree on w within the step-size resolution."""
    d = to_dev(tiny)
    prm = P.default_params(tiny["step"])
    w, st = P.solve_projection(d["f0"], None, d["U"], d["y"], tiny["vol"], tiny["cb"], np.zeros(3), prm)
    wo, sto, _ = O.solve_projection(tiny["f0"], None, tiny["U"], tiny["y"], tiny["vol"], tiny["cb"],
                                    np.zeros(3), prm)
    assert 1 <= st["iters"] <= 10 and st["evals"] >= st["iters"] + 1
    assert np.linalg.norm(w - wo) < 0.05, (w, wo, st, sto)
    # warm start at the oracle's answer: at most a few small steps
    w2, st2 = P.solve_projection(d["f0"], None, d["U"], d["y"], tiny["vol"], tiny["cb"], wo, prm)
    assert np.linalg.norm(w2 - wo) < 0.05


def test_solve_recovers_intensity_scaling(P):
    pb = make_problem((40, 40, 24, 4.0, 4.0, 4.0), 3, (64, 48, 4.0, 4.0), 0.6, (0.5, -0.3, 0.2),
                      noise=0.0, seeds=(31, 32, 33), scale_ab=(1.3, 0.2))
    d = to_dev(pb)
    prm = P.default_params(pb["step"], mu_min=1e-6, max_iter=60, max_trials=40)
    w, st = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    assert abs(st["a"] - 1.3) < 2e-3 and abs(st["b"] - 0.2) < 2e-3
    assert np.linalg.norm(w - pb["w_true"]) < 5e-3


def test_solve_singular_and_zero_iterations(P, tiny):
    d = to_dev(tiny)
    y = torch.full_like(d["y"], 1.0)
    with pytest.raises(P.PcasError) as e:
        P.solve_projection(d["f0"], None, d["U"], y, tiny["vol"], tiny["cb"], np.zeros(3),
                           P.default_params(tiny["step"]))
    assert e.value.code == P.SINGULAR
    w, st = P.solve_projection(d["f0"], None, d["U"], d["y"], tiny["vol"], tiny["cb"], np.full(3, 0.1),
                               P.default_params(tiny["step"], max_iter=0))
    assert st["iters"] == 0 and st["evals"] == 1 and np.allclose(w, 0.1)


# ------------------------------------------------------------ localisation
def test_localize_matches_oracle(P):
    vol = S.volume(64, 64, 32, 4.0, 4.0, 4.0)
    U = S.eigen_dvfs(vol, 3, seed=2)
    mean = (0.2 * U[1]).astype(np.float32)
    tU, tm = torch.from_numpy(U.ravel()).cuda(), torch.from_numpy(mean.ravel()).cuda()
    for w, c_ref in [((1.2, -0.4, 0.3), (20.0, -5.0, 10.0)), ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
                     ((-1.5, 1.0, 0.5), (-60.0, 30.0, -20.0))]:
        c, ok = P.localize_tumor(tm, tU, np.array(w), vol, np.array(c_ref))
        co, oko = O.localize_tumor(mean, U, np.array(w), vol, np.array(c_ref))
        assert ok == oko and np.abs(c - co).max() <= 1e-4


# -------------------------------------------- the sequence workload at full size
@pytest.fixture(scope="module")
def sequence_problem():
    s = SEQUENCE
    w_true = S.breathing_trace(s["n_proj"], s["fps"], s["period"], s["amp"], K=3)[17]
    angle = S.gantry_angles(s["n_proj"])[17]
    return make_problem(s["vol"], s["K"], s["det"], angle, w_true, noise=0.01, seeds=s["seeds"],
                        tumor=s["tumor"])


def test_sequence_size_drr_sampled(P, sequence_problem):
    """Full-size warp + DRR: sampled rays against the oracle one ray at a time."""
    pb = sequence_problem
    d = to_dev(pb)
    w = pb["w_true"] * 0.8
    f = P.warp_volume(d["f0"], P.pca_dvf(None, d["U"], w, pb["vol"]), pb["vol"])
    p = np32(P.drr_forward(f, pb["vol"], pb["cb"], pb["step"]))
    fo = O.warp_volume(pb["f0"], O.pca_dvf(None, pb["U"], w, pb["vol"]), pb["vol"])
    g = S.rng(40)
    nu, nv = pb["cb"]["nu"], pb["cb"]["nv"]
    idx = [(int(g.integers(nu)), int(g.integers(nv))) for _ in range(150)] + [(0, 0), (nu - 1, nv - 1)]
    ref = np.array([O.drr_ray(fo, pb["vol"], pb["cb"], pb["step"], iu, iv) for iu, iv in idx])
    got = np.array([p[iv * nu + iu] for iu, iv in idx])
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(p).max()


def test_sequence_size_cost_grad(P, sequence_problem):
    """Full size, the kernels the solver runs (fused warp, solver DRR, residual,
    fused adjoint gradient) against the oracle's full evaluation."""
    pb = sequence_problem
    d = to_dev(pb)
    w = pb["w_true"] * 0.5
    J, G, ab = P.cost_grad(d["f0"], None, d["U"], w, d["y"], pb["vol"], pb["cb"], pb["step"])
    Jo, Go, abo = O.cost_grad(pb["f0"], None, pb["U"], w, pb["y"], pb["vol"], pb["cb"], pb["step"])
    assert abs(J - Jo) <= 1e-4 * Jo
    assert np.linalg.norm(G - Go) <= 1e-3 * np.linalg.norm(Go), (G, Go)


def test_sequence_size_solve_properties(P, sequence_problem):
    pb = sequence_problem
    d = to_dev(pb)
    prm = P.default_params(pb["step"])
    w, st = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], np.zeros(3), prm)
    # the cost falls to the energy of the 1 % noise added to y (a ~ 1)
    sigma = 0.01 * np.abs(pb["y"]).max() / 1.01
    M = pb["cb"]["nu"] * pb["cb"]["nv"]
    assert st["J"] < st["J0"] and st["J"] <= 1.3 * M * sigma**2, (st, M * sigma**2)
    c, ok = P.localize_tumor(None, d["U"], w, pb["vol"], pb["c_ref"])
    ct, _ = O.localize_tumor(None, pb["U"], pb["w_true"], pb["vol"], pb["c_ref"])
    assert ok and np.linalg.norm(c - ct) < 1.0, (w, pb["w_true"], c, ct)


def test_sequence_size_solve_matches_oracle(P, sequence_problem):
    """One projection of the sequence workload at full size (256x256x100, K = 3,
    512x384), solved by the GPU and by the oracle from the same start: the
    planted coefficients three frames (0.3 s) earlier, a poorer start than the
    Eq. (3) prediction, so that the solve takes several accepted steps with
    different amounts of backtracking before its final rejection.  The same
    iterations and evaluations, w within 2e-3, tumour centroids within 0.05 mm."""
    pb = sequence_problem
    s = SEQUENCE
    trace = S.breathing_trace(s["n_proj"], s["fps"], s["period"], s["amp"], K=3)
    w0 = trace[14]
    d = to_dev(pb)
    prm = P.default_params(pb["step"])
    w, st = P.solve_projection(d["f0"], None, d["U"], d["y"], pb["vol"], pb["cb"], w0, prm)
    wo, sto, _ = O.solve_projection(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], w0, prm)
    assert sto["iters"] >= 3
    assert (st["iters"], st["evals"]) == (sto["iters"], sto["evals"]), (st, sto)
    assert np.abs(w - wo).max() < 2e-3, (w, wo)
    assert abs(st["J"] - sto["J"]) <= 1e-4 * sto["J"], (st, sto)
    c, ok = P.localize_tumor(None, d["U"], w, pb["vol"], pb["c_ref"])
    co, _ = O.localize_tumor(None, pb["U"], wo, pb["vol"], pb["c_ref"])
    print(f"sequence size: |w - w_oracle| = {np.abs(w - wo).max():.2e}, centroid {np.linalg.norm(c - co):.2e} mm "
          f"from the oracle's, iterations {st['iters']}, evaluations {st['evals']}")
    assert ok and np.linalg.norm(c - co) <= 0.05
