"""Pins for the oracle's alternating solve (Appendix, Eq. A.1/A.2 with Armijo),
linear prediction (Eq. 3-5) and tumour localisation (Sec. II.A)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


@pytest.fixture(scope="module")
def problem():
    vol = S.volume(32, 32, 20, 4.0, 4.0, 4.0)
    f0, c_ref = S.phantom(vol, 12.0, seed=1)
    U = S.eigen_dvfs(vol, 3, seed=2)
    cb = S.cone_beam(48, 36, 4.0, 4.0, 0.4)
    return dict(vol=vol, f0=f0, c_ref=c_ref, U=U, cb=cb, step=2.0)


def render(P, U, w):
    f = O.warp_volume(P["f0"], O.pca_dvf(None, U, w, P["vol"]), P["vol"])
    return O.drr_forward(f, P["vol"], P["cb"], P["step"])


def params(step, **kw):
    d = dict(mu0=0.2, alpha=0.1, beta=0.5, mu_min=0.01, max_iter=10, max_trials=30, step=step)
    d.update(kw)
    return d


def test_cost_decreases_monotonically(problem):
    """Appendix: each (A.1) and each accepted Armijo step lowers the cost."""
    P = problem
    y = render(P, P["U"], np.array([0.8, -0.5, 0.3]))
    y = y + S.gaussian_noise(y.shape, 0.01 * y.max(), 3, np.float64)
    w, st, trace = O.solve_projection(P["f0"], None, P["U"], y, P["vol"], P["cb"], np.zeros(3), params(P["step"]))
    assert st["iters"] >= 3
    assert np.all(np.diff(trace) <= 0), trace
    assert trace[-1] < 0.2 * trace[0]


def test_recovers_planted_coefficients_noise_free(problem):
    P = problem
    w_true = np.array([0.5, -0.3, 0.2])
    y = render(P, P["U"], w_true)
    w, st, _ = O.solve_projection(P["f0"], None, P["U"], y, P["vol"], P["cb"], np.zeros(3),
                                  params(P["step"], mu_min=1e-8, max_iter=60, max_trials=40))
    assert np.linalg.norm(w - w_true) < 1e-6, (w, st)
    assert abs(st["a"] - 1.0) < 1e-6 and abs(st["b"]) < 1e-6


def test_recovers_rigid_translation(problem):
    """Sec. II.A: three eigenvectors span all 3D translations; with u_k = 10 mm e_k
    the coefficients are the shift in cm, including the depth component."""
    P = problem
    Ut = S.translation_dvfs(P["vol"], 3)
    w_true = np.array([0.3, 0.15, -0.2])
    y = render(P, Ut, w_true)
    w, st, _ = O.solve_projection(P["f0"], None, Ut, y, P["vol"], P["cb"], np.zeros(3),
                                  params(P["step"], mu_min=1e-8, max_iter=100, max_trials=40))
    assert np.linalg.norm(w - w_true) < 1e-5, (w, st)


def test_intensity_scaling_recovered(problem):
    """Eq. (2): the measured image may differ from the DRR by y -> (P f - b) / a."""
    P = problem
    w_true = np.array([0.5, -0.3, 0.2])
    y = (render(P, P["U"], w_true) - 0.2) / 1.3
    w, st, _ = O.solve_projection(P["f0"], None, P["U"], y, P["vol"], P["cb"], np.zeros(3),
                                  params(P["step"], mu_min=1e-8, max_iter=60, max_trials=40))
    assert abs(st["a"] - 1.3) < 1e-5 and abs(st["b"] - 0.2) < 1e-5
    assert np.linalg.norm(w - w_true) < 1e-5


def test_stopping_rules(problem):
    """Appendix: stop after max_iter iterations, or when no mu >= mu_min passes."""
    P = problem
    y = render(P, P["U"], np.array([0.5, -0.3, 0.2]))
    w, st, trace = O.solve_projection(P["f0"], None, P["U"], y, P["vol"], P["cb"], np.zeros(3),
                                      params(P["step"], max_iter=2))
    assert st["iters"] == 2 and len(trace) == 3
    # at the optimum no trial step can pass: the solve stops without moving
    w_true = np.array([0.5, -0.3, 0.2])
    w2, st2, _ = O.solve_projection(P["f0"], None, P["U"], y, P["vol"], P["cb"], w_true, params(P["step"]))
    assert st2["iters"] <= 1 and np.allclose(w2, w_true, atol=1e-12)
    # evaluations = 1 initial render + trials; trials per iteration are bounded by the mu schedule
    mu_sched = [0.2 * 0.5**j for j in range(30) if 0.2 * 0.5**j >= 0.01]
    assert st["evals"] <= 1 + 2 * len(mu_sched)


def test_paper_constants_are_the_defaults_scaled():
    """Appendix constants (mu0=2, alpha=0.1, beta=0.5, mu_min=0.1, 10 iterations) assume
    w with standard deviation 10; the synthetic w are O(1), so mu0 and mu_min scale by 1/10."""
    A = GOLDEN["armijo"]
    assert (A["mu0"], A["alpha"], A["beta"], A["mu_min"], A["max_iter"]) == (2.0, 0.1, 0.5, 0.1, 10)
    p = params(1.0)
    assert p["mu0"] == A["mu0"] / A["w_std_preconditioned"] and p["mu_min"] == A["mu_min"] / A["w_std_preconditioned"]


# ------------------------------------------------------------------ Eq. (3)-(5)
def test_lp_fit_sinusoid_closed_form():
    """A sampled sinusoid obeys w(t) = 2 cos(omega dt) w(t-1) - w(t-2) exactly."""
    fps = 10.0
    t = np.arange(200) / fps
    periods = [4.0, 3.0]
    trace = np.stack([np.sin(2 * math.pi * t / T + 0.3) for T in periods], 1)
    c = O.lp_fit(trace, 2)
    for k, T in enumerate(periods):
        assert abs(c[k, 0] - 2 * math.cos(2 * math.pi / (T * fps))) < 1e-9
        assert abs(c[k, 1] + 1.0) < 1e-9


@pytest.mark.parametrize("key", ["eq4_digital_phantom", "eq5_physical_phantom"])
def test_lp_fit_reproduces_paper_coefficients(key):
    """A damped oscillation r^t cos(theta t) has exactly the order-2 predictor
    (2 r cos theta, -r^2); building one from each printed row of Eq. (4)/(5) and
    fitting it must return the printed numbers."""
    rows = np.array(GOLDEN[key]["c"])
    T = 120
    t = np.arange(T)
    cols = []
    for c1, c2 in rows:
        r = math.sqrt(-c2)
        th = math.acos(c1 / (2 * r))
        cols.append(r**t * np.cos(th * t + 0.4))
    c = O.lp_fit(np.stack(cols, 1), GOLDEN["prediction_order"]["L"])
    np.testing.assert_allclose(c, rows, atol=1e-9)


def test_lp_predict_extrapolates_sinusoid():
    fps, T = 10.7, 3.4
    t = np.arange(50) / fps
    w = np.sin(2 * math.pi * t / T)[:, None]
    c = O.lp_fit(w[:40], 2)
    for n in range(42, 50):
        pred = O.lp_predict(np.array([[w[n - 1, 0]], [w[n - 2, 0]]]), c)
        assert abs(pred[0] - w[n, 0]) < 1e-9


def test_lp_physical_phantom_rate_plausible():
    """Eq. (5) at the 10.7 Hz projection rate of Sec. II.C implies a lightly damped
    oscillation with a breathing-like period."""
    c1, c2 = GOLDEN["eq5_physical_phantom"]["c"][0]
    r = math.sqrt(-c2)
    th = math.acos(c1 / (2 * r))
    period = 2 * math.pi / th / GOLDEN["eq5_physical_phantom"]["rate_hz"]
    assert 0.99 < r < 1.0 and 2.5 < period < 6.5


# ------------------------------------------------------------- localisation
def test_localize_uniform_translation():
    vol = S.volume(20, 20, 16, 4.0, 4.0, 4.0)
    N = 20 * 20 * 16
    tau = np.array([3.0, -2.0, 5.0])
    mean = np.repeat(-tau[:, None], N, 1)
    c_ref = np.array([4.0, -6.0, 2.0])
    c, ok = O.localize_tumor(mean, np.zeros((0, 3, N)), np.zeros(0), vol, c_ref)
    assert ok and np.allclose(c, c_ref + tau, atol=1e-12)


def test_localize_linear_field_closed_form():
    """x(X) = A X is reproduced exactly by trilinear interpolation inside the grid,
    so the fixed point of c + A c = c_ref is (I + A)^-1 c_ref."""
    vol = S.volume(24, 22, 20, 3.0, 3.0, 3.0)
    x = vol["ox"] + 3.0 * np.arange(24); y = vol["oy"] + 3.0 * np.arange(22); z = vol["oz"] + 3.0 * np.arange(20)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    A = np.array([[0.05, 0.02, -0.03], [0.01, -0.04, 0.02], [0.03, 0.01, 0.06]])
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    U = (A @ pts)[None]                      # one eigenvector, w = 1
    c_ref = np.array([5.0, -7.0, 4.0])
    c, ok = O.localize_tumor(None, U, np.array([1.0]), vol, c_ref, max_iter=200, tol_mm=1e-12)
    assert ok
    np.testing.assert_allclose(c, np.linalg.solve(np.eye(3) + A, c_ref), atol=1e-9)


def test_localize_smooth_field_solves_the_fixed_point_equation():
    """A smooth random motion (three eigenvector fields, w ~ O(1)): the
    returned point satisfies c + x(c) = c_ref, with x(c) evaluated
    independently by scipy's linear interpolation of the field (zero outside
    the grid), and agrees with a general root finder started elsewhere."""
    nd = pytest.importorskip("scipy.ndimage")
    opt = pytest.importorskip("scipy.optimize")
    vol = S.volume(40, 36, 28, 3.0, 3.0, 3.0)
    U = S.eigen_dvfs(vol, 3, seed=9).astype(np.float64)
    w = np.array([0.8, -0.5, 0.3])
    dvf = np.tensordot(w, U, axes=(0, 0)).reshape(3, 28, 36, 40)     # mm, [c][z][y][x]
    o = np.array([vol["ox"], vol["oy"], vol["oz"]])
    s = np.array([vol["sx"], vol["sy"], vol["sz"]])

    def x_of(c):
        q = (np.asarray(c) - o) / s                                      # voxel index (x, y, z)
        coords = np.array([[q[2]], [q[1]], [q[0]]])
        return np.array([nd.map_coordinates(dvf[k], coords, order=1, mode="constant", cval=0.0)[0]
                         for k in range(3)])

    for c_ref in (np.array([6.0, -4.0, 3.0]), np.array([-15.0, 10.0, -8.0])):
        c, ok = O.localize_tumor(None, U, w, vol, c_ref, max_iter=500, tol_mm=1e-12)
        assert ok
        assert np.abs(c + x_of(c) - c_ref).max() <= 1e-9
        sol = opt.root(lambda v: v + x_of(v) - c_ref, c_ref + 2.0, method="hybr", tol=1e-13)
        assert sol.success
        np.testing.assert_allclose(c, sol.x, atol=1e-7)


def test_localize_reports_non_convergence():
    vol = S.volume(24, 22, 20, 3.0, 3.0, 3.0)
    U = S.eigen_dvfs(vol, 1, seed=4)
    c, ok = O.localize_tumor(None, U, np.array([1.0]), vol, np.zeros(3), max_iter=1, tol_mm=1e-12)
    assert not ok
