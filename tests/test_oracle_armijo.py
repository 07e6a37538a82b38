"""Pins for the oracle's line search (Appendix, the paragraph after Eq. A.2):
d = -G/||G||, step sizes mu0, beta mu0, beta^2 mu0, ... tried from mu0 at every
iteration, the first mu with J(w + mu d) <= J(w) - alpha mu ||G|| (a, b held)
accepted, and, when no mu >= mu_min passes, no step taken and the solve ended.

Two independent routes:

* the oracle's per-iteration record on a K = 3 problem, every decision in it
  re-derived from separate evaluations (warp, projector, cost at held a, b);
* a K = 1 problem on which the warped volume is exactly affine in w, so J along
  d is a known quadratic, J(w + mu d) = J - mu ||G|| + mu^2 ||P h||^2, and the
  whole trajectory follows in closed form on the host.
"""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S


def params(step, **kw):
    d = dict(mu0=0.2, alpha=0.1, beta=0.5, mu_min=0.01, max_iter=10, max_trials=30, step=step)
    d.update(kw)
    return d


def schedule(prm):
    """The step sizes one iteration may try: mu0 beta^j >= mu_min, at most max_trials."""
    mus, mu = [], prm["mu0"]
    while mu >= prm["mu_min"] and len(mus) < prm["max_trials"]:
        mus.append(mu)
        mu *= prm["beta"]
    return mus


# ------------------------------------------------------------ K = 3 record
@pytest.fixture(scope="module")
def problem():
    vol = S.volume(32, 32, 20, 4.0, 4.0, 4.0)
    f0, _ = S.phantom(vol, 12.0, seed=1)
    U = S.eigen_dvfs(vol, 3, seed=2)
    cb = S.cone_beam(48, 36, 4.0, 4.0, 0.4)
    return dict(vol=vol, f0=f0, U=U, cb=cb, step=2.0)


def render(P, w):
    f = O.warp_volume(P["f0"], O.pca_dvf(None, P["U"], w, P["vol"]), P["vol"])
    return O.drr_forward(f, P["vol"], P["cb"], P["step"])


def check_record(P, y, w_init, prm):
    """Re-derives every iteration of the oracle's record; returns the record."""
    w_out, st, rows = O.solve_projection_log(P["f0"], None, P["U"], y, P["vol"], P["cb"], w_init, prm)
    mus = schedule(prm)
    w = np.array(w_init, dtype=np.float64)
    for it, r in enumerate(rows):
        # the iterate is the previous one moved by the accepted step
        assert np.array_equal(r["w"], w), (it, r["w"], w)
        # (A.1) at the iterate, then the gradient with (a, b) held
        J, G, (a, b) = O.cost_grad(P["f0"], None, P["U"], w, y, P["vol"], P["cb"], P["step"])
        assert abs(r["J"] - J) <= 1e-12 * J and abs(r["a"] - a) <= 1e-12 * abs(a)
        assert abs(r["b"] - b) <= 1e-12 * max(abs(b), 1.0)
        assert np.allclose(r["G"], G, rtol=1e-12, atol=1e-14 * np.abs(G).max())
        gn = float(np.sqrt(np.sum(G * G)))
        assert abs(r["gnorm"] - gn) <= 1e-12 * gn
        assert np.allclose(r["d"], -G / gn, rtol=1e-12, atol=1e-15)
        # mu restarts at mu0: the trials of this iteration are the schedule's head
        n = r["trials"]
        assert 1 <= n <= len(mus)
        for j in range(n):
            Jt = O.cost(render(P, w + mus[j] * r["d"]), y, a, b)
            passes = Jt <= r["J"] - prm["alpha"] * mus[j] * r["gnorm"]
            if j < n - 1:
                assert not passes, (it, j, "a larger step size passed but was not taken")
            else:
                assert passes == r["accepted"], (it, j, passes, r["accepted"])
        if r["accepted"]:
            assert r["mu"] == mus[n - 1]
            w = w + r["mu"] * r["d"]
        else:
            # no mu >= mu_min passed: no step and the solve ends here
            assert n == len(mus) and r["mu"] == 0.0
            assert it == len(rows) - 1
    assert np.array_equal(w_out, w)
    assert st["iters"] == len(rows)
    assert st["evals"] == 1 + sum(r["trials"] for r in rows)
    return rows, st


def test_record_reproduced_from_separate_evaluations(problem):
    P = problem
    y = render(P, np.array([0.8, -0.5, 0.3]))
    y = y + S.gaussian_noise(y.shape, 0.01 * y.max(), 3, np.float64)
    prm = params(P["step"])
    rows, st = check_record(P, y, np.zeros(3), prm)
    # the case exercises backtracking after long steps and the final rejection
    assert any(r["accepted"] and r["trials"] == 1 for r in rows)
    assert any(r["accepted"] and r["trials"] >= 2 for r in rows)
    assert not rows[-1]["accepted"] and st["iters"] < prm["max_iter"]


def test_record_with_trial_cap(problem):
    """max_trials caps the schedule of an iteration (the tiny workload's form)."""
    P = problem
    y = render(P, np.array([0.5, -0.3, 0.2]))
    prm = params(P["step"], mu_min=0.0, max_trials=3, max_iter=6)
    rows, _ = check_record(P, y, np.zeros(3), prm)
    assert all(r["trials"] <= 3 for r in rows)


# ------------------------------------------------- K = 1, closed form
def affine_problem():
    """f0 linear in the voxel indices and one eigenvector moving only the
    interior voxels along z.  Trilinear interpolation reproduces a linear
    function exactly and no tap leaves the grid, so warp(f0, w) = f0 + w h with
    h = (df0/dk) (10 mm / sz) on the interior: P f(w) = p0 + w p1 exactly."""
    vol = S.volume(24, 24, 16, 4.0, 4.0, 4.0)
    nx, ny, nz = vol["nx"], vol["ny"], vol["nz"]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f0 = (0.01 + 0.002 * i + 0.001 * j + 0.003 * k).astype(np.float64)
    interior = (i >= 3) & (i <= nx - 4) & (j >= 3) & (j <= ny - 4) & (k >= 3) & (k <= nz - 4)
    U = np.zeros((1, 3) + f0.shape)
    U[0, 2] = 10.0 * interior
    h = 0.003 * (10.0 / vol["sz"]) * interior
    cb = S.cone_beam(40, 30, 4.0, 4.0, 0.3)
    return vol, f0.ravel(), U.reshape(1, 3, -1), h.ravel(), cb


def closed_form_solve(p0, p1, y, w0, prm):
    """The Appendix loop with J along d from its quadratic: per iteration
    (a, b) by least squares of p(w) on (y, 1), r = p - a y - b, G = 2 <r, p1>,
    d = -sign(G), and J(w + mu d) = J - mu |G| + mu^2 <p1, p1>."""
    c = float(p1 @ p1)
    A = np.stack([y, np.ones_like(y)], axis=1)
    w, rows, evals = w0, [], 1
    for _ in range(prm["max_iter"]):
        p = p0 + w * p1
        (a, b), *_ = np.linalg.lstsq(A, p, rcond=None)
        r = p - a * y - b
        J, G = float(r @ r), 2.0 * float(r @ p1)
        gn = abs(G)
        if gn == 0.0:
            break
        d = -G / gn
        mu, tried, acc = prm["mu0"], 0, False
        while tried < prm["max_trials"] and mu >= prm["mu_min"]:
            tried += 1
            Jt = J - mu * gn + mu * mu * c
            bound = J - prm["alpha"] * mu * gn
            assert abs(Jt - bound) > 1e-7 * J, "decision too close to call"
            if Jt <= bound:
                acc = True
                break
            mu *= prm["beta"]
        evals += tried
        rows.append(dict(w=w, J=J, gnorm=gn, d=d, mu=mu if acc else 0.0, trials=tried, accepted=acc))
        if not acc:
            break
        w = w + mu * d
    return w, rows, evals


@pytest.mark.parametrize("w_true,mu0,y_scale", [(0.27, 0.2, (1.0, 0.0)), (-0.33, 0.2, (1.3, 0.2)),
                                                (0.19, 0.35, (0.8, -0.1))])
def test_affine_k1_trajectory_in_closed_form(w_true, mu0, y_scale):
    vol, f0, U, h, cb = affine_problem()
    step = 2.0
    # the premise: the warp is affine in w over the range the solve visits
    for w in (-0.4, 0.15, 0.4):
        f = O.warp_volume(f0, O.pca_dvf(None, U, np.array([w]), vol), vol)
        assert np.abs(f - (f0 + w * h)).max() <= 1e-15
    p0 = O.drr_forward(f0, vol, cb, step)
    p1 = O.drr_forward(h, vol, cb, step)
    a_t, b_t = y_scale
    y = (p0 + w_true * p1 - b_t) / a_t
    prm = params(step, mu0=mu0, mu_min=1e-3, max_iter=12)
    w_cf, rows_cf, evals_cf = closed_form_solve(p0, p1, y, 0.0, prm)
    w_o, st, rows = O.solve_projection_log(f0, None, U, y, vol, cb, np.zeros(1), prm)
    assert len(rows) == len(rows_cf) and st["iters"] == len(rows_cf)
    assert st["evals"] == evals_cf
    for r, q in zip(rows, rows_cf):
        assert abs(r["w"][0] - q["w"]) <= 1e-12
        assert abs(r["J"] - q["J"]) <= 1e-9 * q["J"] + 1e-15
        assert abs(r["gnorm"] - q["gnorm"]) <= 1e-9 * q["gnorm"]
        assert r["d"][0] == q["d"]
        assert (r["accepted"], r["trials"], r["mu"]) == (q["accepted"], q["trials"], q["mu"])
    assert abs(w_o[0] - w_cf) <= 1e-12
    # the trajectory backtracks by different amounts from one iteration to the next
    assert len({q["trials"] for q in rows_cf}) >= 2
