"""FP64 CPU oracle for the single-projection PCA motion solve (Li et al.,
arXiv:1102.1712).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product package
``paper_1102_1712_gb300`` never does.  The arithmetic lives in ``oracle.c``
(plain C, double precision, one function per definition of the paper); this
module only compiles it with gcc and marshals numpy arrays through ctypes.

Parity status of each routine (what pins it is in ``tests/test_oracle_*.py``):
  pca_dvf, warp_volume, trilinear, trilinear_grad, drr_forward, drr_ray,
  siddon_forward, siddon_ray, drr_adjoint, intensity_fit, cost, cost_grad, grad_forward_mode,
  warp_adjoint, cost_grad_f0, solve_projection, solve_projection_log, localize_tumor, lp_fit,
  lp_predict -- all pinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
             "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


class Vol(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("sx", C.c_double), ("sy", C.c_double), ("sz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class CB(C.Structure):
    _fields_ = [("sad", C.c_double), ("sdd", C.c_double), ("nu", C.c_int), ("nv", C.c_int),
                ("du", C.c_double), ("dv", C.c_double), ("off_u", C.c_double),
                ("off_v", C.c_double), ("angle", C.c_double)]


class Params(C.Structure):
    _fields_ = [("mu0", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("mu_min", C.c_double), ("max_iter", C.c_int), ("max_trials", C.c_int),
                ("step", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("evals", C.c_int), ("status", C.c_int),
                ("J0", C.c_double), ("J", C.c_double), ("a", C.c_double),
                ("b", C.c_double), ("mu_last", C.c_double)]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            for name, res, args in [
                ("oracle_pca_dvf", C.c_int, [_D, _D, C.c_int, _D, C.POINTER(Vol), _D]),
                ("oracle_warp_volume", C.c_int, [_D, _D, C.POINTER(Vol), _D]),
                ("oracle_trilinear", C.c_double, [_D, C.POINTER(Vol), C.c_double, C.c_double, C.c_double]),
                ("oracle_trilinear_grad", None, [_D, C.POINTER(Vol), C.c_double, C.c_double, C.c_double, _D]),
                ("oracle_drr_forward", C.c_int, [_D, C.POINTER(Vol), C.POINTER(CB), C.c_double, _D]),
                ("oracle_drr_ray", C.c_double, [_D, C.POINTER(Vol), C.POINTER(CB), C.c_double, C.c_int, C.c_int]),
                ("oracle_drr_adjoint", C.c_int, [_D, C.POINTER(Vol), C.POINTER(CB), C.c_double, _D]),
                ("oracle_siddon_forward", C.c_int, [_D, C.POINTER(Vol), C.POINTER(CB), _D]),
                ("oracle_siddon_ray", C.c_double, [_D, C.POINTER(Vol), C.POINTER(CB), C.c_int, C.c_int]),
                ("oracle_intensity_fit", C.c_int, [_D, _D, C.c_long, _D, _D]),
                ("oracle_cost", C.c_double, [_D, _D, C.c_long, C.c_double, C.c_double]),
                ("oracle_cost_grad", C.c_int, [_D, _D, _D, C.c_int, _D, _D, C.POINTER(Vol), C.POINTER(CB),
                                               C.c_double, C.c_int, _D, _D, _D]),
                ("oracle_grad_forward_mode", C.c_int, [_D, _D, _D, C.c_int, _D, _D, C.POINTER(Vol),
                                                       C.POINTER(CB), C.c_double, C.c_double, C.c_double, _D]),
                ("oracle_warp_adjoint", C.c_int, [_D, _D, C.POINTER(Vol), _D]),
                ("oracle_cost_grad_f0", C.c_int, [_D, _D, _D, C.c_int, _D, _D, C.POINTER(Vol), C.POINTER(CB),
                                                  C.c_double, C.c_int, _D, _D, _D]),
                ("oracle_solve_projection", C.c_int, [_D, _D, _D, C.c_int, _D, C.POINTER(Vol), C.POINTER(CB),
                                                      _D, C.POINTER(Params), _D, C.POINTER(Stats), _D]),
                ("oracle_solve_projection_log", C.c_int, [_D, _D, _D, C.c_int, _D, C.POINTER(Vol),
                                                          C.POINTER(CB), _D, C.POINTER(Params), _D,
                                                          C.POINTER(Stats), _D, _D]),
                ("oracle_localize_tumor", C.c_int, [_D, _D, C.c_int, _D, C.POINTER(Vol), _D, C.c_int,
                                                    C.c_double, _D]),
                ("oracle_lp_fit", C.c_int, [_D, C.c_int, C.c_int, C.c_int, _D]),
                ("oracle_lp_predict", C.c_int, [_D, _D, C.c_int, C.c_int, _D]),
            ]:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _d(a):
    """Contiguous float64 copy (or view) of an array, kept alive by the caller."""
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def vol_struct(v: dict) -> Vol:
    return Vol(v["nx"], v["ny"], v["nz"], v["sx"], v["sy"], v["sz"], v["ox"], v["oy"], v["oz"])


def cb_struct(g: dict) -> CB:
    return CB(g["sad"], g["sdd"], g["nu"], g["nv"], g["du"], g["dv"],
              g.get("off_u", 0.0), g.get("off_v", 0.0), g["angle"])


def _nvox(v):
    return v["nx"] * v["ny"] * v["nz"]


def _check(rc, what):
    if rc not in (0,):
        raise RuntimeError(f"oracle {what} returned status {rc}")


def pca_dvf(mean, U, w, vol):
    N = _nvox(vol)
    U = _d(U).reshape(-1, 3, N)
    K = U.shape[0]
    mean = None if mean is None else _d(mean).reshape(3, N)
    w = _d(w)
    out = np.empty((3, N))
    _check(lib().oracle_pca_dvf(_p(mean), _p(U), K, _p(w), C.byref(vol_struct(vol)), _p(out)), "pca_dvf")
    return out


def warp_volume(f0, dvf, vol):
    f0 = _d(f0).ravel()
    dvf = _d(dvf).reshape(3, -1)
    out = np.empty_like(f0)
    _check(lib().oracle_warp_volume(_p(f0), _p(dvf), C.byref(vol_struct(vol)), _p(out)), "warp_volume")
    return out


def trilinear(f, vol, q):
    f = _d(f).ravel()
    return lib().oracle_trilinear(_p(f), C.byref(vol_struct(vol)), float(q[0]), float(q[1]), float(q[2]))


def trilinear_grad(f, vol, q):
    f = _d(f).ravel()
    d = np.zeros(3)
    lib().oracle_trilinear_grad(_p(f), C.byref(vol_struct(vol)), float(q[0]), float(q[1]), float(q[2]), _p(d))
    return d


def drr_forward(f, vol, cb, step):
    f = _d(f).ravel()
    p = np.empty(cb["nu"] * cb["nv"])
    _check(lib().oracle_drr_forward(_p(f), C.byref(vol_struct(vol)), C.byref(cb_struct(cb)),
                                    float(step), _p(p)), "drr_forward")
    return p


def drr_ray(f, vol, cb, step, iu, iv):
    f = _d(f).ravel()
    return lib().oracle_drr_ray(_p(f), C.byref(vol_struct(vol)), C.byref(cb_struct(cb)),
                                float(step), int(iu), int(iv))


def siddon_forward(f, vol, cb):
    """Exact line integrals of the piecewise-constant volume (Sec. II.B)."""
    f = _d(f).ravel()
    p = np.empty(cb["nu"] * cb["nv"])
    _check(lib().oracle_siddon_forward(_p(f), C.byref(vol_struct(vol)), C.byref(cb_struct(cb)), _p(p)),
           "siddon_forward")
    return p


def siddon_ray(f, vol, cb, iu, iv):
    f = _d(f).ravel()
    return lib().oracle_siddon_ray(_p(f), C.byref(vol_struct(vol)), C.byref(cb_struct(cb)), int(iu), int(iv))


def drr_adjoint(img, vol, cb, step):
    img = _d(img).ravel()
    g = np.empty(_nvox(vol))
    _check(lib().oracle_drr_adjoint(_p(img), C.byref(vol_struct(vol)), C.byref(cb_struct(cb)),
                                    float(step), _p(g)), "drr_adjoint")
    return g


def intensity_fit(p, y):
    p, y = _d(p).ravel(), _d(y).ravel()
    a, b = C.c_double(), C.c_double()
    rc = lib().oracle_intensity_fit(_p(p), _p(y), p.size, C.byref(a), C.byref(b))
    if rc == 2:
        raise np.linalg.LinAlgError("Y^T Y singular")
    _check(rc, "intensity_fit")
    return a.value, b.value


def cost(p, y, a, b):
    p, y = _d(p).ravel(), _d(y).ravel()
    return lib().oracle_cost(_p(p), _p(y), p.size, float(a), float(b))


def cost_grad(f0, mean, U, w, y, vol, cb, step, ab=None):
    """Returns (J, G, (a, b)); (a, b) from Eq. (A.1) unless given."""
    N = _nvox(vol)
    f0 = _d(f0).ravel()
    U = _d(U).reshape(-1, 3, N)
    K = U.shape[0]
    mean = None if mean is None else _d(mean).reshape(3, N)
    w, y = _d(w), _d(y).ravel()
    abv = np.zeros(2) if ab is None else _d(ab).copy()
    J = C.c_double()
    G = np.zeros(K)
    _check(lib().oracle_cost_grad(_p(f0), _p(mean), _p(U), K, _p(w), _p(y), C.byref(vol_struct(vol)),
                                  C.byref(cb_struct(cb)), float(step), 1 if ab is None else 0,
                                  _p(abv), C.byref(J), _p(G)), "cost_grad")
    return J.value, G, (abv[0], abv[1])


def warp_adjoint(z, dvf, vol):
    z = _d(z).ravel()
    dvf = _d(dvf).reshape(3, -1)
    out = np.empty_like(z)
    _check(lib().oracle_warp_adjoint(_p(z), _p(dvf), C.byref(vol_struct(vol)), _p(out)), "warp_adjoint")
    return out


def cost_grad_f0(f0, mean, U, w, y, vol, cb, step, ab=None):
    """Returns (J, dJ/df0 (N,), (a, b)) at fixed w; (a, b) from Eq. (A.1) unless given."""
    N = _nvox(vol)
    f0 = _d(f0).ravel()
    U = _d(U).reshape(-1, 3, N)
    K = U.shape[0]
    mean = None if mean is None else _d(mean).reshape(3, N)
    w, y = _d(w), _d(y).ravel()
    abv = np.zeros(2) if ab is None else _d(ab).copy()
    J = C.c_double()
    out = np.zeros(N)
    _check(lib().oracle_cost_grad_f0(_p(f0), _p(mean), _p(U), K, _p(w), _p(y), C.byref(vol_struct(vol)),
                                     C.byref(cb_struct(cb)), float(step), 1 if ab is None else 0, _p(abv),
                                     C.byref(J), _p(out)), "cost_grad_f0")
    return J.value, out, (abv[0], abv[1])


def grad_forward_mode(f0, mean, U, w, y, vol, cb, step, a, b):
    N = _nvox(vol)
    f0 = _d(f0).ravel()
    U = _d(U).reshape(-1, 3, N)
    K = U.shape[0]
    mean = None if mean is None else _d(mean).reshape(3, N)
    w, y = _d(w), _d(y).ravel()
    G = np.zeros(K)
    _check(lib().oracle_grad_forward_mode(_p(f0), _p(mean), _p(U), K, _p(w), _p(y),
                                          C.byref(vol_struct(vol)), C.byref(cb_struct(cb)),
                                          float(step), float(a), float(b), _p(G)), "grad_forward_mode")
    return G


def solve_projection(f0, mean, U, y, vol, cb, w_init, params: dict):
    """Returns (w_out, stats dict, J trace)."""
    N = _nvox(vol)
    f0 = _d(f0).ravel()
    U = _d(U).reshape(-1, 3, N)
    K = U.shape[0]
    mean = None if mean is None else _d(mean).reshape(3, N)
    y, w0 = _d(y).ravel(), _d(w_init)
    prm = Params(params["mu0"], params["alpha"], params["beta"], params["mu_min"],
                 params["max_iter"], params["max_trials"], params["step"])
    w_out = np.zeros(K)
    st = Stats()
    trace = np.full(params["max_iter"] + 1, np.nan)
    rc = lib().oracle_solve_projection(_p(f0), _p(mean), _p(U), K, _p(y), C.byref(vol_struct(vol)),
                                       C.byref(cb_struct(cb)), _p(w0), C.byref(prm), _p(w_out),
                                       C.byref(st), _p(trace))
    _check(rc, "solve_projection")
    stats = {k: getattr(st, k) for k, _ in Stats._fields_}
    return w_out, stats, trace[: stats["iters"] + 1]


def solve_projection_log(f0, mean, U, y, vol, cb, w_init, params: dict):
    """solve_projection with a record of every iteration that reached the line
    search: a list of dicts with J, a, b (at the iterate, after Eq. A.1), gnorm,
    mu (the accepted step size, 0.0 if none), trials, accepted, and the
    iterate w, gradient G and direction d."""
    N = _nvox(vol)
    f0 = _d(f0).ravel()
    U = _d(U).reshape(-1, 3, N)
    K = U.shape[0]
    mean = None if mean is None else _d(mean).reshape(3, N)
    y, w0 = _d(y).ravel(), _d(w_init)
    prm = Params(params["mu0"], params["alpha"], params["beta"], params["mu_min"],
                 params["max_iter"], params["max_trials"], params["step"])
    w_out = np.zeros(K)
    st = Stats()
    trace = np.full(params["max_iter"] + 1, np.nan)
    stride = 7 + 3 * K
    log = np.full((max(params["max_iter"], 1), stride), np.nan)
    rc = lib().oracle_solve_projection_log(_p(f0), _p(mean), _p(U), K, _p(y), C.byref(vol_struct(vol)),
                                           C.byref(cb_struct(cb)), _p(w0), C.byref(prm), _p(w_out),
                                           C.byref(st), _p(trace), _p(log))
    _check(rc, "solve_projection_log")
    stats = {k: getattr(st, k) for k, _ in Stats._fields_}
    rows = []
    for r in log:
        if np.isnan(r[0]):
            break
        rows.append(dict(J=r[0], a=r[1], b=r[2], gnorm=r[3], mu=r[4], trials=int(r[5]), accepted=bool(r[6]),
                         w=r[7:7 + K].copy(), G=r[7 + K:7 + 2 * K].copy(), d=r[7 + 2 * K:7 + 3 * K].copy()))
    return w_out, stats, rows


def localize_tumor(mean, U, w, vol, c_ref, max_iter=50, tol_mm=1e-6):
    N = _nvox(vol)
    U = _d(U).reshape(-1, 3, N)
    K = U.shape[0]
    mean = None if mean is None else _d(mean).reshape(3, N)
    w, c_ref = _d(w), _d(c_ref)
    out = np.zeros(3)
    rc = lib().oracle_localize_tumor(_p(mean), _p(U), K, _p(w), C.byref(vol_struct(vol)), _p(c_ref),
                                     int(max_iter), float(tol_mm), _p(out))
    if rc not in (0, 4):
        _check(rc, "localize_tumor")
    return out, rc == 0


def lp_fit(trace, L):
    trace = _d(trace)
    T, K = trace.shape
    c = np.zeros((K, L))
    _check(lib().oracle_lp_fit(_p(trace), T, K, L, _p(c)), "lp_fit")
    return c


def lp_predict(hist, c):
    """hist[l-1] = w*(t-l), shape (L, K); c shape (K, L)."""
    hist, c = _d(hist), _d(c)
    L, K = hist.shape
    w0 = np.zeros(K)
    _check(lib().oracle_lp_predict(_p(hist), _p(c), K, L, _p(w0)), "lp_predict")
    return w0
