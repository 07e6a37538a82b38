"""The seeded input generators: reproducible, shaped and scaled as stated."""
import numpy as np

from paper_1102_1712_gb300 import synth as S


def test_phantom_reproducible_and_structured():
    vol = S.volume(64, 64, 32, 4.0, 4.0, 4.0)
    a, ca = S.phantom(vol, 15.0, seed=1)
    b, cb = S.phantom(vol, 15.0, seed=1)
    c, _ = S.phantom(vol, 15.0, seed=2)
    assert a.dtype == np.float32 and a.shape == (32, 64, 64)
    assert np.array_equal(a, b) and np.array_equal(ca, cb) and not np.array_equal(a, c)
    assert set(np.unique(a)) <= {0.0, np.float32(0.005), np.float32(0.02)}
    # the tumour centre voxel carries tumour attenuation and is surrounded by lung
    i = np.round((ca - [vol["ox"], vol["oy"], vol["oz"]]) / 4.0).astype(int)
    assert a[i[2], i[1], i[0]] == np.float32(0.02)
    assert (a == np.float32(0.005)).sum() > 0.05 * a.size


def test_eigen_dvf_scaling():
    vol = S.volume(40, 36, 24, 4.0, 4.0, 4.0)
    U = S.eigen_dvfs(vol, 3, seed=2)
    assert U.shape == (3, 3, 40 * 36 * 24) and U.dtype == np.float32
    assert abs(np.abs(U[0, 2]).max() - 10.0) < 1e-4          # u_1: 10 mm peak SI
    for k in (1, 2):
        assert abs(np.abs(U[k]).max() - 10.0) < 1e-4
    assert np.array_equal(U, S.eigen_dvfs(vol, 3, seed=2))


def test_breathing_trace_regular_and_irregular():
    W = S.breathing_trace(600, 10.0, period_s=4.0, amp_mm=15.0, K=3)
    assert W.shape == (600, 3)
    assert abs(W[:, 0].max() - 1.5) < 1e-3 and W[:, 0].min() > -1e-9
    np.testing.assert_allclose(W[40:, 0], W[:-40, 0], atol=1e-12)        # period 4 s at 10 fps
    Wi = S.breathing_trace(600, 10.0, irregular=True, drift_mm=3.0, seed=11)
    assert not np.allclose(Wi, W)
    assert abs(Wi[-1, 0] - Wi[0, 0]) < 2.5


def test_angles_and_noise():
    a = S.gantry_angles(600, 360.0)
    assert a.shape == (600,) and abs(a[1] - a[0] - np.deg2rad(0.6)) < 1e-12
    n = S.gaussian_noise((1000,), 0.5, seed=3)
    assert n.dtype == np.float32 and 0.4 < n.std() < 0.6
