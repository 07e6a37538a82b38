"""Pins of the oracle's Siddon projector (exact radiological path through the
piecewise-constant voxels, Sec. II.B): closed-form chords through a uniform
box and through a single voxel cube, an axis-aligned ray along a column of
voxel centres, and a brute-force fine Riemann sum on a random volume."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S


def frame(cb):
    a = cb["angle"]
    Sx = np.array([cb["sad"] * np.sin(a), -cb["sad"] * np.cos(a), 0.0])
    ew = np.array([-np.sin(a), np.cos(a), 0.0])
    eu = np.array([np.cos(a), np.sin(a), 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    return Sx, ew, eu, ev


def ray(cb, iu, iv):
    Sx, ew, eu, ev = frame(cb)
    u = (iu - 0.5 * (cb["nu"] - 1)) * cb["du"] + cb["off_u"]
    v = (iv - 0.5 * (cb["nv"] - 1)) * cb["dv"] + cb["off_v"]
    d = cb["sdd"] * ew + u * eu + v * ev
    return Sx, d / np.linalg.norm(d)


def chord(Sx, d, lo, hi):
    """Length of the ray S + t d (t >= 0) inside the box [lo, hi] (slab method)."""
    t0, t1 = 0.0, np.inf
    for c in range(3):
        if d[c] == 0.0:
            if not (lo[c] <= Sx[c] <= hi[c]):
                return 0.0
            continue
        a, b = (lo[c] - Sx[c]) / d[c], (hi[c] - Sx[c]) / d[c]
        t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
    return max(t1 - t0, 0.0)


def box_of(vol):
    o = np.array([vol["ox"], vol["oy"], vol["oz"]])
    s = np.array([vol["sx"], vol["sy"], vol["sz"]])
    n = np.array([vol["nx"], vol["ny"], vol["nz"]])
    return o, s, n


def test_uniform_volume_gives_the_chord():
    vol = S.volume(13, 11, 7, 3.0, 2.5, 4.0)
    cb = S.cone_beam(24, 18, 3.0, 3.0, 0.7, off_u=2.0, off_v=-1.5)
    mu = 0.02
    p = O.siddon_forward(np.full(13 * 11 * 7, mu), vol, cb).reshape(18, 24)
    o, s, n = box_of(vol)
    hits = 0
    for iv in range(18):
        for iu in range(24):
            Sx, d = ray(cb, iu, iv)
            L = chord(Sx, d, o - 0.5 * s, o + (n - 0.5) * s)
            assert abs(p[iv, iu] - mu * L) <= 1e-12 * max(1.0, mu * L), (iu, iv)
            hits += L > 0
    assert hits > 100


@pytest.mark.parametrize("angle", [0.3, 1.9, 4.1])
def test_single_voxel_gives_its_cube_chord(angle):
    vol = S.volume(9, 8, 6, 4.0, 3.0, 5.0)
    o, s, n = box_of(vol)
    g = S.rng(5)
    for _ in range(4):
        i, j, k = (int(g.integers(0, n[c])) for c in range(3))
        f = np.zeros((6, 8, 9))
        f[k, j, i] = 1.0
        centre = o + np.array([i, j, k]) * s
        cb = S.cone_beam(15, 15, 0.9, 0.9, angle)
        # aim the detector so that its middle rays cross the chosen voxel
        Sx, ew, eu, ev = frame(cb)
        rel = centre - Sx
        scale = cb["sdd"] / rel.dot(ew)
        cb["off_u"], cb["off_v"] = rel.dot(eu) * scale, rel.dot(ev) * scale
        p = O.siddon_forward(f, vol, cb).reshape(15, 15)
        crossed = 0
        for iv in range(15):
            for iu in range(15):
                Sx, d = ray(cb, iu, iv)
                L = chord(Sx, d, centre - 0.5 * s, centre + 0.5 * s)
                assert abs(p[iv, iu] - L) <= 1e-12 * max(1.0, L)
                crossed += L > 0
        assert crossed > 10


def test_axis_aligned_ray_sums_a_column():
    vol = S.volume(7, 10, 5, 2.0, 3.0, 2.5)           # odd nx, nz: a voxel column on the central ray
    f = S.rng(6).uniform(0.0, 1.0, (5, 10, 7))
    cb = S.cone_beam(9, 7, 1.0, 1.0, 0.0)             # angle 0: central ray along +y through x = z = 0
    p = O.siddon_ray(f, vol, cb, 4, 3)
    assert abs(p - 3.0 * f[2, :, 3].sum()) <= 1e-12 * p


def test_matches_a_fine_riemann_sum():
    vol = S.volume(6, 5, 4, 4.0, 4.0, 4.0)
    f = S.rng(7).uniform(0.0, 1.0, (4, 5, 6))
    cb = S.cone_beam(6, 5, 6.0, 6.0, 2.6, off_u=1.3, off_v=0.7)
    o, s, n = box_of(vol)
    h = 2e-3
    for iu, iv in [(1, 1), (2, 3), (4, 2), (3, 0)]:
        Sx, d = ray(cb, iu, iv)
        t = np.arange(cb["sad"] - 40.0, cb["sad"] + 40.0, h) + 0.5 * h
        X = Sx[None, :] + t[:, None] * d[None, :]
        idx = np.floor((X - o) / s + 0.5).astype(int)
        ok = np.all((idx >= 0) & (idx < n), axis=1)
        ref = h * f[idx[ok, 2], idx[ok, 1], idx[ok, 0]].sum()
        got = O.siddon_ray(f, vol, cb, iu, iv)
        assert ref > 1.0 and abs(got - ref) <= 3e-3 * ref, (iu, iv, got, ref)


def test_rays_that_miss_are_zero():
    vol = S.volume(8, 8, 8, 2.0, 2.0, 2.0)
    cb = S.cone_beam(4, 4, 1.0, 1.0, 0.5, off_u=400.0)
    assert np.all(O.siddon_forward(np.ones(512), vol, cb) == 0.0)
