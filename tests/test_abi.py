"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/pcasolve.h declares, rejects invalid arguments
before touching the device, and its host-only routines (Eq. 3) agree with the
oracle."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1102_1712_gb300 import build as B
from paper_1102_1712_gb300 import pcasolve as P
from paper_1102_1712_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.lib()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", text, re.M):
            names.append(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    for must in ["pca_dvf", "warp_volume", "drr_forward", "drr_adjoint", "cost_grad",
                 "solve_projection", "localize_tumor", "lp_fit", "lp_predict",
                 "pcas_workspace_bytes", "pcas_last_error", "pcas_version"]:
        assert must in names
    for n in names:
        assert hasattr(lib, n), n
    assert lib.pcas_version() == 1


def test_binding_exposes_the_same_names():
    for n in ["pca_dvf", "warp_volume", "drr_forward", "drr_adjoint", "cost_grad",
              "solve_projection", "localize_tumor", "lp_fit", "lp_predict"]:
        assert callable(getattr(P, n))


def test_workspace_bytes_host_only(lib):
    vol = S.volume(256, 256, 100, 2.0, 2.0, 2.5)
    cb = S.cone_beam(512, 384, 0.776, 0.776)
    n = P.workspace_bytes(vol, cb, 3)
    npad = (((256 + 6) + 3) // 4 * 4) * 260 * 104          # two-voxel zero halo
    M = 512 * 384
    cap = 32 * 32 * 25 * 256                                 # 8x8x4 tiles of the Jacobian compaction
    f0h = 262 * 262 * 106 * 4                                # reference CT with a three-voxel zero halo
    occ = 65 * 65 * 26 * 4 + 33 * 33 * 13                   # bricks: 4^3 of the solver volumes, 8^3 of f0
    need = f0h + occ + npad * (4 + 8 + 16) + M * (6 * 4 + 36) + cap * (4 + 4 * 3)   # f (+ 5th), its pairs, 4 cands,
    assert need <= n < need + 2_000_000 and n % 256 == 0       # 6 projections, ray table, compacted voxels
    assert P.workspace_bytes(vol, cb, 0) == 0 and P.workspace_bytes(vol, cb, 9) == 0
    # room for the y-fastest layout too: a non-square grid takes the larger of the two
    v2 = S.volume(200, 300, 50, 2.0, 2.0, 2.0)
    pa = ((200 + 9) // 4 * 4) * 304 * 54
    pb = ((300 + 9) // 4 * 4) * 204 * 54
    assert P.workspace_bytes(v2, cb, 3) >= max(pa, pb) * (4 + 16)


def test_volume_size_limits(lib):
    """32-bit voxel offsets: ny, nz <= 65535 and the halo layout below 2^31 elements."""
    cb = S.cone_beam(64, 48, 1.0, 1.0)
    assert P.workspace_bytes(S.volume(8, 65536, 4, 1, 1, 1), cb, 1) == 0
    assert P.workspace_bytes(S.volume(8, 4, 65536, 1, 1, 1), cb, 1) == 0
    assert P.workspace_bytes(S.volume(1300, 1300, 1260, 1, 1, 1), cb, 1) == 0   # (1310)(1304)(1264) > 2^31
    assert P.workspace_bytes(S.volume(20000, 20000, 1, 1, 1, 1), cb, 1) == 0    # halo copy: 20006^2 7 > 2^31
    assert P.workspace_bytes(S.volume(1024, 1024, 1024, 1, 1, 1), cb, 1) > 0


FAKE = C.c_void_p(0x1000)    # never dereferenced: every call below fails its host checks


def _vol(**kw):
    v = dict(S.volume(16, 16, 8, 2.0, 2.0, 2.0)); v.update(kw); return P.vol_struct(v)


def _cb(**kw):
    g = dict(S.cone_beam(32, 24, 1.5, 1.5, 0.3)); g.update(kw); return P.cb_struct(g)


@pytest.mark.parametrize("vol,cb,step", [
    (_vol(nx=0), _cb(), 1.0),
    (_vol(sx=-1.0), _cb(), 1.0),
    (_vol(), _cb(nu=0), 1.0),
    (_vol(), _cb(du=0.0), 1.0),
    (_vol(), _cb(), 0.0),
    (_vol(), _cb(), float("nan")),
    (_vol(), _cb(sad=10.0, sdd=20.0), 1.0),            # volume not in front of the source
    (_vol(ox=float("inf")), _cb(), 1.0),
])
def test_invalid_geometry_rejected_before_launch(lib, vol, cb, step):
    rc = lib.drr_forward(FAKE, C.byref(vol), C.byref(cb), step, FAKE, None)
    assert rc == P.INVALID_ARG and P.last_error()
    rc = lib.drr_adjoint(FAKE, C.byref(vol), C.byref(cb), step, FAKE, None)
    assert rc == P.INVALID_ARG


def test_invalid_model_and_workspace_rejected(lib):
    vol, cb = _vol(), _cb()
    w = np.zeros(8)
    D = C.POINTER(C.c_double)
    J = C.c_double()
    G = np.zeros(8)
    ab = np.zeros(2)
    assert lib.pca_dvf(None, FAKE, 0, w.ctypes.data_as(D), C.byref(vol), FAKE, None) == P.INVALID_ARG
    assert lib.pca_dvf(None, FAKE, 9, w.ctypes.data_as(D), C.byref(vol), FAKE, None) == P.INVALID_ARG
    assert lib.pca_dvf(None, None, 3, w.ctypes.data_as(D), C.byref(vol), FAKE, None) == P.INVALID_ARG
    bad = w.copy(); bad[1] = np.nan
    assert lib.pca_dvf(None, FAKE, 3, bad.ctypes.data_as(D), C.byref(vol), FAKE, None) == P.INVALID_ARG
    need = lib.pcas_workspace_bytes(C.byref(vol), C.byref(cb), 3)
    args = (FAKE, None, FAKE, 3, w.ctypes.data_as(D), FAKE, C.byref(vol), C.byref(cb), 1.0,
            C.byref(J), G.ctypes.data_as(D), ab.ctypes.data_as(D))
    assert lib.cost_grad(*args, C.c_void_p(0x100000), need - 1, None) == P.INVALID_ARG
    assert "too small" in P.last_error()
    assert lib.cost_grad(*args, C.c_void_p(0x100010), need, None) == P.INVALID_ARG
    assert "aligned" in P.last_error()
    assert lib.cost_grad(*args, None, need, None) == P.INVALID_ARG
    prm = P.params_struct(P.default_params(1.0, beta=1.5))
    st = P.Stats()
    wo = np.zeros(3)
    assert lib.solve_projection(FAKE, None, FAKE, 3, FAKE, C.byref(vol), C.byref(cb), w.ctypes.data_as(D),
                                C.byref(prm), wo.ctypes.data_as(D), C.byref(st), C.c_void_p(0x100000),
                                need, None) == P.INVALID_ARG
    c = np.zeros(3)
    assert lib.localize_tumor(None, FAKE, 3, w.ctypes.data_as(D), C.byref(vol), c.ctypes.data_as(D), 0,
                              1e-6, c.ctypes.data_as(D), None) == P.INVALID_ARG


def test_lp_fit_and_predict_match_oracle(lib):
    W = S.breathing_trace(300, 10.0, irregular=True, seed=5)
    for L in (1, 2, 3):
        np.testing.assert_allclose(P.lp_fit(W, L), O.lp_fit(W, L), rtol=1e-10, atol=1e-12)
    c = O.lp_fit(W, 2)
    hist = W[[9, 8]]
    np.testing.assert_allclose(P.lp_predict(hist, c), O.lp_predict(hist, c), rtol=1e-14, atol=1e-15)
    with pytest.raises(P.PcasError):
        P.lp_fit(W[:4], 2)
    t = np.arange(100) / 10.0
    c = P.lp_fit(np.sin(2 * math.pi * t / 4.0)[:, None], 2)
    assert abs(c[0, 0] - 2 * math.cos(2 * math.pi / 40)) < 1e-9 and abs(c[0, 1] + 1) < 1e-9


def test_tuning_table_host_only(lib):
    """The launch-shape table is host state: set / get / clear and the checks."""
    vol = S.volume(64, 64, 32, 4.0, 4.0, 4.0)
    cb = S.cone_beam(128, 96, 3.1, 3.1)
    P.tuning_clear()
    d = P.tuning_get(vol, cb, 3)
    assert d == dict(ray_lw1=3, chunk1=0, voxel_tile=0, gather_per_sm=8, skip_empty=1, ray_lw4=[3] * 8,
                     chunk=[16] * 8, swap=[0, 0, 0, 1, 1, 1, 0, 0])
    t = dict(ray_lw1=2, chunk1=64, voxel_tile=5, gather_per_sm=2, skip_empty=0, ray_lw4=[2, 3, 4, 2, 3, 4, 2, 3],
             chunk=[12, 16, 24, 2, 64, 12, 16, 24], swap=[0, 1] * 4)
    P.tuning_set(vol, cb, 3, t)
    assert P.tuning_get(vol, cb, 3) == t
    assert P.tuning_get(S.volume(60, 64, 32, 4.0, 4.0, 4.0), cb, 3) == t        # same bucket (x in 33..64)
    assert P.tuning_get(S.volume(96, 64, 32, 4.0, 4.0, 4.0), cb, 3) == d        # next bucket
    assert P.tuning_get(vol, cb, 5) == d and P.tuning_get(vol, cb, 3, dtype=P.BF16) == d
    for bad in (dict(t, ray_lw1=5), dict(t, chunk1=-2), dict(t, chunk1=33), dict(t, chunk1=130),
                dict(t, voxel_tile=6), dict(t, gather_per_sm=0), dict(t, gather_per_sm=27),
                dict(t, skip_empty=2), dict(t, skip_empty=-1),
                dict(t, ray_lw4=[1] + [3] * 7), dict(t, chunk=[13] + [16] * 7), dict(t, chunk=[0] * 8),
                dict(t, chunk=[66] * 8), dict(t, swap=[2] + [0] * 7)):
        with pytest.raises(P.PcasError):
            P.tuning_set(vol, cb, 3, bad)
    P.tuning_clear()
    assert P.tuning_get(vol, cb, 3) == d


def test_static_scratch_example_fits(lib):
    """The size the header quotes as fitting the static scratch does fit."""
    n = P.workspace_bytes(S.volume(72, 72, 40, 4.0, 4.0, 4.0), S.cone_beam(192, 144, 2.0, 2.0), 3)
    assert 0 < n <= 16 * 1024 * 1024
