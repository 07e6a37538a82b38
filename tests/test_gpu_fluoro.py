"""Fixed-angle (fluoroscopy) variant: every frame of a breathing sequence is
projected at one gantry angle, so the projection geometry is constant.  One
device-driven solver is built once and reused for every frame; each frame is
warm-started by the Eq. (3) prediction.  Measured images come from Siddon's
projector (no inverse crime)."""
import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import synth as S

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


def test_fixed_angle_sequence(P):
    vol = S.volume(61, 53, 29, 4.0, 3.5, 4.5)
    f0, c_ref = S.phantom(vol, 14.0, seed=61)
    U = S.eigen_dvfs(vol, 3, seed=62)
    fps, n = 10.0, 14
    trace = S.breathing_trace(n, fps, period_s=4.0, amp_mm=12.0, K=3)
    train = S.breathing_trace(200, fps, period_s=4.0, amp_mm=12.0, K=3, t0=-30.0)
    cb = S.cone_beam(101, 77, 3.5, 3.5, np.deg2rad(75.0))
    step = 0.5 * min(vol["sx"], vol["sy"], vol["sz"])
    prm = P.default_params(step)
    tf0, tU = torch.from_numpy(f0.ravel()).cuda(), torch.from_numpy(U.ravel()).cuda()
    c_lp = P.lp_fit(train, 2)
    sv = P.Solver(tf0, None, tU, vol, cb, prm)
    hist, errs = [], []
    for t in range(n):
        f = O.warp_volume(f0, O.pca_dvf(None, U, trace[t], vol), vol)
        y = O.siddon_forward(f, vol, cb)
        y = (y + S.gaussian_noise(y.shape, 0.01 * np.abs(y).max(), seed=600 + t, dtype=np.float64))
        yd = torch.from_numpy(y.astype(np.float32)).cuda()
        w0 = np.zeros(3) if t == 0 else (hist[-1] if t == 1 else P.lp_predict(np.stack([hist[-1], hist[-2]]), c_lp))
        w, st = sv.solve(yd, w0)
        wh, sth = P.solve_projection(tf0, None, tU, yd, vol, cb, w0, prm)
        assert np.array_equal(w, wh) and st == sth, t
        hist.append(w)
        c, _ = P.localize_tumor(None, tU, w, vol, c_ref)
        ct, _ = O.localize_tumor(None, U, trace[t], vol, c_ref)
        errs.append(np.linalg.norm(c - ct))
    errs = np.array(errs)
    print(f"fixed-angle sequence: centroid error mean {errs.mean():.3f} mm, max {errs.max():.3f} mm")
    assert errs[2:].mean() < 1.0 and errs.max() < 2.5
    sv.close()


def test_fixed_view_cache_is_bitwise_the_uncached_solve(P):
    """Sec. IV: with the gantry held still the projection matrix is constant;
    the solver's cache of P^T's per-voxel footprints and ray weights for that
    view gives bitwise the same solves as computing them in every gradient
    (host-driven solve, device-driven solve and a run of projections), solves
    at other angles are unaffected, and turning the cache off restores the
    uncached path."""
    vol = S.volume(61, 53, 29, 4.0, 3.5, 4.5)
    f0, c_ref = S.phantom(vol, 14.0, seed=61)
    U = S.eigen_dvfs(vol, 3, seed=62)
    fps, n = 10.0, 8
    trace = S.breathing_trace(n, fps, period_s=4.0, amp_mm=12.0, K=3)
    train = S.breathing_trace(200, fps, period_s=4.0, amp_mm=12.0, K=3, t0=-30.0)
    ang = np.deg2rad(75.0)
    cb = S.cone_beam(101, 77, 3.5, 3.5, ang, off_u=2.0)
    step = 0.5 * min(vol["sx"], vol["sy"], vol["sz"])
    prm = P.default_params(step)
    tf0, tU = torch.from_numpy(f0.ravel()).cuda(), torch.from_numpy(U.ravel()).cuda()
    ys = []
    for t in range(n):
        y = O.siddon_forward(O.warp_volume(f0, O.pca_dvf(None, U, trace[t], vol), vol), vol, cb)
        y = y + S.gaussian_noise(y.shape, 0.01 * np.abs(y).max(), seed=700 + t, dtype=np.float64)
        ys.append(torch.from_numpy(y.astype(np.float32)).cuda())
    c_lp = P.lp_fit(train, 2)
    plain = P.Solver(tf0, None, tU, vol, cb, prm)
    cached = P.Solver(tf0, None, tU, vol, cb, prm)
    nbytes = cached.fix_view(ang)
    assert nbytes > 4 * vol["nx"] * vol["ny"] * vol["nz"]
    for t in (0, 3, 7):
        w0 = 0.5 * trace[t]
        wa, sa = plain.solve(ys[t], w0)
        wb, sb = cached.solve(ys[t], w0)
        assert np.array_equal(wa, wb) and sa == sb, t
    # runs of projections: warm start and localisation on the device
    plain.seq_begin(c_lp, c_ref)
    cached.seq_begin(c_lp, c_ref)
    ra = plain.solve_sequence(ys, [ang] * n, w_first=np.zeros(3))
    rb = cached.solve_sequence(ys, [ang] * n, w_first=np.zeros(3))
    for t, ((wa, sa, ca, _), (wb, sb, cbb, _)) in enumerate(zip(ra, rb)):
        assert np.array_equal(wa, wb) and sa == sb and np.array_equal(ca, cbb), t
    # another angle: the cache is not used, the results are the plain solver's
    yo = torch.from_numpy(O.siddon_forward(O.warp_volume(f0, O.pca_dvf(None, U, trace[2], vol), vol), vol,
                                           dict(cb, angle=0.3)).astype(np.float32)).cuda()
    wa, sa = plain.solve(yo, np.zeros(3), angle=0.3)
    wb, sb = cached.solve(yo, np.zeros(3), angle=0.3)
    assert np.array_equal(wa, wb) and sa == sb
    # off again, then a cache that is too small is refused
    cached.fix_view(None)
    wb, sb = cached.solve(ys[3], 0.5 * trace[3])
    wa, sa = plain.solve(ys[3], 0.5 * trace[3])
    assert np.array_equal(wa, wb) and sa == sb
    small = torch.empty(4096, dtype=torch.uint8, device="cuda")
    ptr = (small.data_ptr() + 255) & ~255
    rc = P.lib().pcas_solver_fix_view(cached.h, float(ang), ptr, 2048, P._stream(None))
    assert rc == P.INVALID_ARG
    plain.close()
    cached.close()
