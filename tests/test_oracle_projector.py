"""Pins for the oracle's cone-beam projector P (Eq. 2) and its transpose P^T
(gradient formula below Eq. A.2): closed-form line integrals, the projection
geometry, convergence under refinement and the adjoint identity."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S


def ray(cb, iu, iv):
    """Source and unit direction of pixel (iu, iv) in the stated view convention."""
    th = cb["angle"]
    Sx = np.array([cb["sad"] * math.sin(th), -cb["sad"] * math.cos(th), 0.0])
    ew = np.array([-math.sin(th), math.cos(th), 0.0])
    eu = np.array([math.cos(th), math.sin(th), 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    u = (iu - 0.5 * (cb["nu"] - 1)) * cb["du"] + cb["off_u"]
    v = (iv - 0.5 * (cb["nv"] - 1)) * cb["dv"] + cb["off_v"]
    P = Sx + cb["sdd"] * ew + u * eu + v * ev
    d = P - Sx
    return Sx, d / np.linalg.norm(d)


def gaussian_blob(vol, c, sigma, A=1.0):
    x, y, z = (vol["ox"] + vol["sx"] * np.arange(vol["nx"]), vol["oy"] + vol["sy"] * np.arange(vol["ny"]),
               vol["oz"] + vol["sz"] * np.arange(vol["nz"]))
    gx = np.exp(-((x - c[0]) ** 2) / (2 * sigma**2))
    gy = np.exp(-((y - c[1]) ** 2) / (2 * sigma**2))
    gz = np.exp(-((z - c[2]) ** 2) / (2 * sigma**2))
    return A * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]


def test_axis_aligned_ray_is_column_sum():
    """A ray along +y through voxel centres with step | s_y sees the piecewise-linear
    interpolant at its nodes: the Riemann sum is the exact integral s_y * sum_j f."""
    vol = S.volume(5, 8, 3, 2.0, 2.0, 2.0)            # centre voxel column i=2, k=1 lies on x=z=0
    f0 = S.rng(1).uniform(0.5, 1.5, (3, 8, 5))
    cb = S.cone_beam(3, 3, 1.0, 1.0, 0.0)             # central pixel (1,1) looks along +y
    p = O.drr_ray(f0, vol, cb, 0.5, 1, 1)
    assert abs(p - 2.0 * f0[1, :, 2].sum()) < 1e-12
    ones = np.ones_like(f0)
    assert abs(O.drr_ray(ones, vol, cb, 0.25, 1, 1) - 8 * 2.0) < 1e-12   # n_y s_y incl. roll-off


@pytest.mark.parametrize("angle", [0.0, 0.6, 2.2])
def test_gaussian_blob_line_integrals_converge_second_order(angle):
    c = np.array([7.0, -5.0, 3.0])
    sig = 10.0
    errs = []
    for s in (4.0, 2.0, 1.0):
        n = int(round(128 / s))
        vol = S.volume(n, n, n, s, s, s)
        f = gaussian_blob(vol, c, sig)
        cb = S.cone_beam(41, 41, 2.0, 2.0, angle)
        e = []
        for iu, iv in [(20, 20), (26, 19), (14, 25), (23, 12), (31, 22)]:
            Sx, dh = ray(cb, iu, iv)
            rel = c - Sx
            dist = np.linalg.norm(rel - (rel @ dh) * dh)
            exact = math.sqrt(2 * math.pi) * sig * math.exp(-dist**2 / (2 * sig**2))
            got = O.drr_ray(f, vol, cb, 0.5 * s, iu, iv)
            e.append(abs(got - exact) / exact)
        errs.append(max(e))
    assert errs[2] < 5e-3, errs
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs   # O(s^2)


def _centroid(img, cb):
    I = img.reshape(cb["nv"], cb["nu"])
    iv, iu = np.mgrid[0:cb["nv"], 0:cb["nu"]]
    return (I * iu).sum() / I.sum(), (I * iv).sum() / I.sum()


@pytest.mark.parametrize("angle,pos,axis_u", [
    (0.0, (30.0, 0.0, -20.0), 0),            # at 0 deg eu = +x
    (math.pi / 2, (0.0, 24.0, 16.0), 1),     # at 90 deg eu = +y
])
def test_blob_projects_to_magnified_position(angle, pos, axis_u):
    """The view convention: a point on the isocentre plane projects with magnification
    sdd/sad along eu (in-plane) and ev = +z."""
    vol = S.volume(64, 64, 64, 2.0, 2.0, 2.0)
    f = gaussian_blob(vol, np.array(pos), 3.0)
    cb = S.cone_beam(121, 101, 1.0, 1.0, angle)
    img = O.drr_forward(f, vol, cb, 1.0)
    cu, cv = _centroid(img, cb)
    mag = cb["sdd"] / cb["sad"]
    assert abs((cu - 60) * cb["du"] - mag * pos[axis_u]) < 0.1
    assert abs((cv - 50) * cb["dv"] - mag * pos[2]) < 0.1


def test_uniform_sphere_chord_lengths():
    R, mu = 30.0, 0.02
    mean_err = []
    for s in (2.0, 1.0):
        n = int(round(100 / s))
        vol = S.volume(n, n, n, s, s, s)
        x = vol["ox"] + s * np.arange(n)
        r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
        f = np.where(r2 <= R * R, mu, 0.0)
        cb = S.cone_beam(61, 61, 1.0, 1.0, 0.3)
        errs = []
        for iu, iv in [(30, 30), (40, 30), (30, 45), (50, 38), (22, 12)]:
            Sx, dh = ray(cb, iu, iv)
            dist = np.linalg.norm(-Sx - ((-Sx) @ dh) * dh)
            exact = mu * 2 * math.sqrt(max(R * R - dist * dist, 0.0))
            err = abs(O.drr_ray(f, vol, cb, 0.5 * s, iu, iv) - exact)
            assert err <= 1.5 * mu * s, (s, iu, iv, err)
            errs.append(err)
        mean_err.append(np.mean(errs))
    assert mean_err[1] < mean_err[0]


@pytest.mark.parametrize("angle,off", [(0.0, (0.0, 0.0)), (0.7, (3.0, -2.0)), (2.5, (-5.0, 4.0))])
def test_adjoint_identity(angle, off):
    """<P x, y> = <x, P^T y> to rounding: P^T is the exact transpose of P."""
    vol = S.volume(13, 11, 9, 3.0, 2.5, 4.0)
    g = S.rng(3)
    x = g.uniform(0, 1, (9, 11, 13))
    cb = S.cone_beam(17, 15, 4.0, 4.5, angle, off_u=off[0], off_v=off[1])
    y = g.uniform(0, 1, 17 * 15)
    step = 0.7
    lhs = O.drr_forward(x, vol, cb, step) @ y
    rhs = x.ravel() @ O.drr_adjoint(y, vol, cb, step)
    assert lhs > 0
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_projector_linear_and_ray_consistent():
    vol = S.volume(12, 10, 8, 3.0, 3.0, 3.0)
    g = S.rng(4)
    a, b = g.uniform(0, 1, (8, 10, 12)), g.uniform(0, 1, (8, 10, 12))
    cb = S.cone_beam(9, 7, 5.0, 5.0, 1.1)
    pa, pb = O.drr_forward(a, vol, cb, 1.5), O.drr_forward(b, vol, cb, 1.5)
    np.testing.assert_allclose(O.drr_forward(2.5 * a + b, vol, cb, 1.5), 2.5 * pa + pb, rtol=1e-13, atol=1e-13)
    assert O.drr_ray(a, vol, cb, 1.5, 4, 3) == pa[3 * 9 + 4]


def test_rays_missing_the_volume_are_zero_and_bad_geometry_rejected():
    vol = S.volume(12, 10, 8, 3.0, 3.0, 3.0)
    f = np.ones((8, 10, 12))
    cb = S.cone_beam(5, 5, 1.0, 1.0, 0.0, off_u=400.0)
    assert np.all(O.drr_forward(f, vol, cb, 1.0) == 0.0)
    with pytest.raises(RuntimeError):
        O.drr_forward(f, vol, S.cone_beam(5, 5, 1.0, 1.0, 0.0, sad=5.0, sdd=50.0), 1.0)   # source inside
    with pytest.raises(RuntimeError):
        O.drr_forward(f, vol, cb, 0.0)
