"""Pins for the oracle's intensity scaling (Eq. A.1), cost (Eq. 2) and gradient
(formula below Eq. A.2)."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S


@pytest.fixture(scope="module")
def problem():
    vol = S.volume(28, 26, 18, 4.0, 4.0, 4.0)
    f0, _ = S.phantom(vol, 12.0, seed=1)
    U = S.eigen_dvfs(vol, 3, seed=2)
    cb = S.cone_beam(40, 30, 4.0, 4.0, 0.4)
    step = 2.0
    w_true = np.array([0.5, -0.3, 0.2])
    f = O.warp_volume(f0, O.pca_dvf(None, U, w_true, vol), vol)
    y_clean = O.drr_forward(f, vol, cb, step)
    return dict(vol=vol, f0=f0, U=U, cb=cb, step=step, w_true=w_true, y_clean=y_clean)


def test_intensity_fit_recovers_exact_affine_relation():
    g = S.rng(5)
    p = g.uniform(0, 3, 500)
    a, b = 1.3, 0.2
    y = (p - b) / a          # then P f = a y + b exactly
    ah, bh = O.intensity_fit(p, y)
    assert abs(ah - a) < 1e-12 and abs(bh - b) < 1e-12
    assert O.cost(p, y, ah, bh) < 1e-24


def test_intensity_fit_is_least_squares():
    g = S.rng(6)
    y = g.uniform(0, 2, 300)
    p = 0.7 * y + 0.1 + 0.05 * g.standard_normal(300)
    a, b = O.intensity_fit(p, y)
    ref = np.linalg.lstsq(np.stack([y, np.ones_like(y)], 1), p, rcond=None)[0]
    assert abs(a - ref[0]) < 1e-12 and abs(b - ref[1]) < 1e-12
    J = O.cost(p, y, a, b)
    for da, db in [(1e-4, 0), (-1e-4, 0), (0, 1e-4), (0, -1e-4)]:
        assert O.cost(p, y, a + da, b + db) > J
    assert abs(J - np.sum((p - a * y - b) ** 2)) < 1e-12 * J


def test_intensity_fit_singular():
    with pytest.raises(np.linalg.LinAlgError):
        O.intensity_fit(np.arange(10.0), np.full(10, 3.0))


def test_cost_and_gradient_vanish_at_planted_w(problem):
    P = problem
    J, G, (a, b) = O.cost_grad(P["f0"], None, P["U"], P["w_true"], P["y_clean"], P["vol"], P["cb"], P["step"])
    assert abs(a - 1) < 1e-12 and abs(b) < 1e-12
    assert J < 1e-20 and np.abs(G).max() < 1e-9


def test_gradient_matches_central_differences(problem):
    P = problem
    w = np.array([0.3, -0.1, 0.05])
    J, G, ab = O.cost_grad(P["f0"], None, P["U"], w, P["y_clean"], P["vol"], P["cb"], P["step"])
    h = 1e-6
    fd = np.zeros(3)
    for k in range(3):
        e = np.zeros(3); e[k] = h
        Jp = O.cost_grad(P["f0"], None, P["U"], w + e, P["y_clean"], P["vol"], P["cb"], P["step"], ab=ab)[0]
        Jm = O.cost_grad(P["f0"], None, P["U"], w - e, P["y_clean"], P["vol"], P["cb"], P["step"], ab=ab)[0]
        fd[k] = (Jp - Jm) / (2 * h)
    assert np.linalg.norm(G) > 0
    assert np.linalg.norm(fd - G) <= 1e-5 * np.linalg.norm(G), (fd, G)


def test_gradient_forward_mode_identity(problem):
    """G_k = 2 <P^T r, h_k> = 2 <r, P h_k>: the adjoint route of the paper and a
    forward projection of the per-voxel sensitivities must agree to rounding."""
    P = problem
    noisy = P["y_clean"] + S.gaussian_noise(P["y_clean"].shape, 0.01 * P["y_clean"].max(), 7, np.float64)
    for w in (np.zeros(3), np.array([0.4, 0.2, -0.3])):
        J, G, (a, b) = O.cost_grad(P["f0"], None, P["U"], w, noisy, P["vol"], P["cb"], P["step"])
        Gf = O.grad_forward_mode(P["f0"], None, P["U"], w, noisy, P["vol"], P["cb"], P["step"], a, b)
        assert np.linalg.norm(G - Gf) <= 1e-10 * np.linalg.norm(G)


def test_cost_grad_with_mean_field(problem):
    """A mean DVF shifts the expansion point: mean + U w == U (w + c) when mean = U c."""
    P = problem
    c = np.array([0.1, 0.2, -0.1])
    mean = np.tensordot(c, P["U"].astype(np.float64), axes=1)
    w = np.array([0.2, -0.1, 0.3])
    J1, G1, _ = O.cost_grad(P["f0"], mean, P["U"], w, P["y_clean"], P["vol"], P["cb"], P["step"])
    J2, G2, _ = O.cost_grad(P["f0"], None, P["U"], w + c, P["y_clean"], P["vol"], P["cb"], P["step"])
    assert abs(J1 - J2) <= 1e-9 * J2
    np.testing.assert_allclose(G1, G2, rtol=1e-8)


# ------------------------------------------- gradient w.r.t. the reference CT
def test_warp_adjoint_identity(problem):
    """<W x, z> = <x, W^T z>: W^T is the exact transpose of the warp (A.5)."""
    P = problem
    dvf = O.pca_dvf(None, P["U"], np.array([0.7, -0.4, 0.5]), P["vol"])
    g = S.rng(12)
    x = g.uniform(0, 1, dvf.shape[1])
    z = g.uniform(0, 1, dvf.shape[1])
    lhs = O.warp_volume(x, dvf, P["vol"]) @ z
    rhs = x @ O.warp_adjoint(z, dvf, P["vol"])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_grad_f0_exact_central_differences(problem):
    """At fixed w and (a, b), J is exactly quadratic in f0 (P and W are linear),
    so a central difference along any direction equals the directional
    derivative up to rounding."""
    P = problem
    w = np.array([0.3, -0.1, 0.05])
    y = P["y_clean"] + S.gaussian_noise(P["y_clean"].shape, 0.01 * P["y_clean"].max(), 13, np.float64)
    J, dJ, ab = O.cost_grad_f0(P["f0"], None, P["U"], w, y, P["vol"], P["cb"], P["step"])
    J2, _, _ = O.cost_grad(P["f0"], None, P["U"], w, y, P["vol"], P["cb"], P["step"])
    assert abs(J - J2) <= 1e-12 * J
    g = S.rng(14)
    f0 = P["f0"].astype(np.float64)
    for _ in range(3):
        dirn = g.standard_normal(f0.shape)
        h = 1e-3
        Jp = O.cost_grad_f0(f0 + h * dirn, None, P["U"], w, y, P["vol"], P["cb"], P["step"], ab=ab)[0]
        Jm = O.cost_grad_f0(f0 - h * dirn, None, P["U"], w, y, P["vol"], P["cb"], P["step"], ab=ab)[0]
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - dJ @ dirn.ravel()) <= 1e-9 * max(abs(fd), 1e-12)
    # single voxels too (the per-voxel check of the differentiation workload)
    flat = f0.ravel()
    for n in g.integers(0, flat.size, 8):
        e = np.zeros_like(flat); e[n] = 1e-2
        Jp = O.cost_grad_f0(flat + e, None, P["U"], w, y, P["vol"], P["cb"], P["step"], ab=ab)[0]
        Jm = O.cost_grad_f0(flat - e, None, P["U"], w, y, P["vol"], P["cb"], P["step"], ab=ab)[0]
        assert abs((Jp - Jm) / 2e-2 - dJ[n]) <= 1e-9 * max(abs(dJ).max(), 1e-12)
