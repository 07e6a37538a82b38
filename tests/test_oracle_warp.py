"""Pins for the oracle's DVF synthesis (Eq. 1), trilinear warp (Eq. A.3/A.5) and
warp Jacobian (Eq. A.8).  Each check uses a property the mathematics fixes, not
a retyping of the oracle's formula."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S


def small_vol(nx=9, ny=7, nz=6, s=(2.0, 3.0, 2.5)):
    return S.volume(nx, ny, nz, *s)


def rand_field(vol, seed, lo=0.0, hi=1.0):
    return S.rng(seed).uniform(lo, hi, (vol["nz"], vol["ny"], vol["nx"]))


def const_dvf(vol, x_mm):
    N = vol["nx"] * vol["ny"] * vol["nz"]
    return np.repeat(np.asarray(x_mm, float)[:, None], N, axis=1)


# ---------------------------------------------------------------- Eq. (1)
def test_pca_dvf_special_cases():
    vol = small_vol()
    N = vol["nx"] * vol["ny"] * vol["nz"]
    g = S.rng(1)
    U = g.standard_normal((4, 3, N))
    mean = g.standard_normal((3, N))
    assert np.array_equal(O.pca_dvf(mean, U, np.zeros(4), vol), mean)          # w = 0 gives the mean
    for k in range(4):                                                        # unit w_k adds u_k
        e = np.zeros(4); e[k] = 1.0
        np.testing.assert_allclose(O.pca_dvf(mean, U, e, vol), mean + U[k], rtol=0, atol=1e-15)
    w1, w2 = g.standard_normal(4), g.standard_normal(4)                       # superposition
    lhs = O.pca_dvf(mean, U, w1 + w2, vol)
    rhs = O.pca_dvf(mean, U, w1, vol) + O.pca_dvf(None, U, w2, vol)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ Eq. (A.3/A.5)
def test_warp_identity_is_exact():
    vol = small_vol()
    f0 = rand_field(vol, 2)
    f = O.warp_volume(f0, const_dvf(vol, [0, 0, 0]), vol)
    assert np.array_equal(f, f0.ravel())


def test_warp_integer_translation_is_index_shift():
    vol = small_vol()
    f0 = rand_field(vol, 3)
    sh = (2, -1, 1)  # voxels along x, y, z
    f = O.warp_volume(f0, const_dvf(vol, [sh[0] * vol["sx"], sh[1] * vol["sy"], sh[2] * vol["sz"]]), vol)
    f = f.reshape(f0.shape)
    ref = np.zeros_like(f0)
    for k in range(vol["nz"]):
        for j in range(vol["ny"]):
            for i in range(vol["nx"]):
                ii, jj, kk = i + sh[0], j + sh[1], k + sh[2]
                if 0 <= ii < vol["nx"] and 0 <= jj < vol["ny"] and 0 <= kk < vol["nz"]:
                    ref[k, j, i] = f0[kk, jj, ii]
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-15)


def test_warp_half_voxel_is_neighbour_mean():
    vol = small_vol()
    f0 = rand_field(vol, 4)
    f = O.warp_volume(f0, const_dvf(vol, [0, 0.5 * vol["sy"], 0]), vol).reshape(f0.shape)
    ref = 0.5 * f0
    ref[:, :-1, :] += 0.5 * f0[:, 1:, :]
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-15)


def test_warp_reproduces_multilinear_functions():
    """Trilinear interpolation is exact for f0 = P(i) Q(j) R(k) with P, Q, R affine;
    this pins every weight and cross term of (A.5)."""
    vol = small_vol(10, 9, 8)
    i = np.arange(vol["nx"]); j = np.arange(vol["ny"]); k = np.arange(vol["nz"])
    P = lambda t: 0.3 + 0.7 * t  # noqa: E731
    Q = lambda t: 1.1 - 0.2 * t  # noqa: E731
    R = lambda t: 0.5 + 0.4 * t  # noqa: E731
    f0 = R(k)[:, None, None] * Q(j)[None, :, None] * P(i)[None, None, :]
    g = S.rng(5)
    N = f0.size
    dvf = np.stack([g.uniform(-1.5, 1.5, N) * vol["sx"], g.uniform(-1.5, 1.5, N) * vol["sy"],
                    g.uniform(-1.5, 1.5, N) * vol["sz"]])
    f = O.warp_volume(f0, dvf, vol)
    kk, jj, ii = np.meshgrid(k, j, i, indexing="ij")
    q1 = ii.ravel() + dvf[0] / vol["sx"]
    q2 = jj.ravel() + dvf[1] / vol["sy"]
    q3 = kk.ravel() + dvf[2] / vol["sz"]
    inside = (q1 >= 0) & (q1 <= vol["nx"] - 1) & (q2 >= 0) & (q2 <= vol["ny"] - 1) & (q3 >= 0) & (q3 <= vol["nz"] - 1)
    assert inside.sum() > N // 4
    np.testing.assert_allclose(f[inside], (P(q1) * Q(q2) * R(q3))[inside], rtol=1e-13, atol=1e-13)


def test_warp_outside_grid_is_zero():
    vol = small_vol()
    f0 = rand_field(vol, 6, 1.0, 2.0)
    f = O.warp_volume(f0, const_dvf(vol, [100 * vol["sx"], 0, 0]), vol)
    assert np.all(f == 0.0)


def test_trilinear_matches_scipy_map_coordinates_order1():
    """Inside the grid, (A.5) is the textbook order-1 spline interpolation."""
    from scipy.ndimage import map_coordinates
    vol = small_vol()
    f0 = rand_field(vol, 7)
    g = S.rng(8)
    for _ in range(50):
        q = g.uniform([0, 0, 0], [vol["nx"] - 1, vol["ny"] - 1, vol["nz"] - 1])
        ref = map_coordinates(f0, [[q[2]], [q[1]], [q[0]]], order=1)[0]
        assert abs(O.trilinear(f0, vol, q) - ref) < 1e-13


# ---------------------------------------------------------------- Eq. (A.8)
def test_jacobian_matches_central_differences_off_grid():
    vol = small_vol()
    f0 = rand_field(vol, 9)
    g = S.rng(10)
    h = 1e-6
    for _ in range(40):
        q = g.uniform([-0.9, -0.9, -0.9], [vol["nx"] - 0.1, vol["ny"] - 0.1, vol["nz"] - 0.1])
        if np.any(np.abs(q - np.round(q)) < 1e-3):
            continue
        d = O.trilinear_grad(f0, vol, q)
        for c in range(3):
            e = np.zeros(3); e[c] = h
            fd = (O.trilinear(f0, vol, q + e) - O.trilinear(f0, vol, q - e)) / (2 * h)
            assert abs(d[c] - fd) < 1e-7, (q, c, d[c], fd)


def test_jacobian_is_right_derivative_on_grid_lines():
    """Appendix, comment after (A.8): at integer q the formula is the right derivative."""
    vol = small_vol()
    f0 = rand_field(vol, 11)
    q = np.array([3.0, 2.0, 4.0])  # exactly on grid lines in every axis
    d = O.trilinear_grad(f0, vol, q)
    h = 1e-7
    for c in range(3):
        e = np.zeros(3); e[c] = h
        right = (O.trilinear(f0, vol, q + e) - O.trilinear(f0, vol, q)) / h
        assert abs(d[c] - right) < 1e-6
    # and on the grid, the right derivative along x is the forward difference
    assert abs(d[0] - (f0[4, 2, 4] - f0[4, 2, 3])) < 1e-15


def test_jacobian_of_multilinear_function():
    vol = small_vol(10, 9, 8)
    i = np.arange(vol["nx"]); j = np.arange(vol["ny"]); k = np.arange(vol["nz"])
    f0 = (0.5 + 0.4 * k)[:, None, None] * (1.1 - 0.2 * j)[None, :, None] * (0.3 + 0.7 * i)[None, None, :]
    q = np.array([3.3, 4.6, 2.2])
    d = O.trilinear_grad(f0, vol, q)
    P, Q, R = 0.3 + 0.7 * q[0], 1.1 - 0.2 * q[1], 0.5 + 0.4 * q[2]
    np.testing.assert_allclose(d, [0.7 * Q * R, -0.2 * P * R, 0.4 * P * Q], rtol=1e-13)
