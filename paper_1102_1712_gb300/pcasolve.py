"""Thin ctypes binding of libpcasolve (include/pcasolve.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device arrays are torch CUDA tensors (float32, contiguous); the
current torch stream is passed to the library.  There is no CPU fallback: if
the library is missing, loading raises.

Names follow the C ABI: pca_dvf, warp_volume, drr_forward, drr_siddon, drr_adjoint,
cost_grad, solve_projection, localize_tumor, lp_fit, lp_predict.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcasolve.so")
KMAX = 8

OK, INVALID_ARG, SINGULAR, CUDA_ERROR, NOT_CONVERGED, TIMEOUT = range(6)
F32, BF16, F16 = range(3)      # storage types of the *_typed calls (pcas_dtype)


class PcasError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pcasolve error {code}: {msg}")
        self.code = code


class Vol(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("sx", C.c_double), ("sy", C.c_double), ("sz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class CB(C.Structure):
    _fields_ = [("sad", C.c_double), ("sdd", C.c_double), ("nu", C.c_int), ("nv", C.c_int),
                ("du", C.c_double), ("dv", C.c_double), ("off_u", C.c_double),
                ("off_v", C.c_double), ("angle_rad", C.c_double)]


class Params(C.Structure):
    _fields_ = [("mu0", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("mu_min", C.c_double), ("max_iter", C.c_int), ("max_trials", C.c_int),
                ("step_mm", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("evals", C.c_int), ("status", C.c_int),
                ("J0", C.c_double), ("J", C.c_double), ("a", C.c_double),
                ("b", C.c_double), ("mu_last", C.c_double)]


class SeqResult(C.Structure):
    """pcas_seq_result: one projection of a run (include/pcasolve.h)."""
    _fields_ = [("w", C.c_double * 8), ("c", C.c_double * 3), ("loc_converged", C.c_int), ("stats", Stats)]


_D = C.POINTER(C.c_double)
_P = C.c_void_p
_lock = threading.Lock()
_lib = None

_SIGS = {
    "pcas_last_error": (C.c_char_p, []),
    "pcas_version": (C.c_int, []),
    "pcas_workspace_bytes": (C.c_size_t, [C.POINTER(Vol), C.POINTER(CB), C.c_int]),
    "pca_dvf": (C.c_int, [_P, _P, C.c_int, _D, C.POINTER(Vol), _P, _P]),
    "warp_volume": (C.c_int, [_P, _P, C.POINTER(Vol), _P, _P]),
    "drr_forward": (C.c_int, [_P, C.POINTER(Vol), C.POINTER(CB), C.c_double, _P, _P]),
    "drr_siddon": (C.c_int, [_P, C.POINTER(Vol), C.POINTER(CB), _P, _P]),
    "drr_adjoint": (C.c_int, [_P, C.POINTER(Vol), C.POINTER(CB), C.c_double, _P, _P]),
    "cost_grad": (C.c_int, [_P, _P, _P, C.c_int, _D, _P, C.POINTER(Vol), C.POINTER(CB), C.c_double,
                            _D, _D, _D, _P, C.c_size_t, _P]),
    "pcas_workspace_bytes_f0": (C.c_size_t, [C.POINTER(Vol), C.POINTER(CB), C.c_int]),
    "cost_grad_f0": (C.c_int, [_P, _P, _P, C.c_int, _D, _P, C.POINTER(Vol), C.POINTER(CB), C.c_double,
                               _D, _D, _D, _P, _P, C.c_size_t, _P]),
    "cost_grad_typed": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, _D, _P, C.POINTER(Vol), C.POINTER(CB),
                                  C.c_double, _D, _D, _D, _P, C.c_size_t, _P]),
    "solve_projection_typed": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, _P, C.POINTER(Vol), C.POINTER(CB), _D,
                                         C.POINTER(Params), _D, C.POINTER(Stats), _P, C.c_size_t, _P]),
    "localize_tumor_typed": (C.c_int, [_P, _P, C.c_int, C.c_int, _D, C.POINTER(Vol), _D, C.c_int,
                                       C.c_double, _D, _P]),
    "cost_grad_static": (C.c_int, [_P, _P, _P, C.c_int, _D, _P, C.POINTER(Vol), C.POINTER(CB),
                                   C.c_double, _D, _D, _D, _P]),
    "solve_projection": (C.c_int, [_P, _P, _P, C.c_int, _P, C.POINTER(Vol), C.POINTER(CB), _D,
                                   C.POINTER(Params), _D, C.POINTER(Stats), _P, C.c_size_t, _P]),
    "localize_tumor": (C.c_int, [_P, _P, C.c_int, _D, C.POINTER(Vol), _D, C.c_int, C.c_double, _D, _P]),
    "lp_fit": (C.c_int, [_D, C.c_int, C.c_int, C.c_int, _D]),
    "lp_predict": (C.c_int, [_D, _D, C.c_int, C.c_int, _D]),
    "pcas_solver_workspace_bytes": (C.c_size_t, [C.POINTER(Vol), C.POINTER(CB), C.c_int]),
    "pcas_solver_create": (C.c_int, [C.POINTER(C.c_void_p), _P, _P, _P, C.c_int, C.c_int, C.POINTER(Vol),
                                     C.POINTER(CB), C.POINTER(Params), _P, C.c_size_t, _P]),
    "pcas_solver_y_buffer": (C.c_void_p, [C.c_void_p]),
    "pcas_solver_solve": (C.c_int, [C.c_void_p, _P, C.c_double, C.c_double, C.c_double, _D, _D,
                                    C.POINTER(Stats), _P]),
    "pcas_solver_destroy": (C.c_int, [C.c_void_p]),
    "pcas_solver_fixed_view_bytes": (C.c_size_t, [C.c_void_p, C.c_double, _P]),
    "pcas_solver_fix_view": (C.c_int, [C.c_void_p, C.c_double, _P, C.c_size_t, _P]),
    "pcas_solver_seq_begin": (C.c_int, [C.c_void_p, _D, C.c_int, _D, C.c_int, C.c_double, _D, C.c_int, _P]),
    "pcas_solver_seq_enqueue": (C.c_int, [C.c_void_p, _P, C.c_double, _D, C.POINTER(C.c_longlong), _P]),
    "pcas_solver_seq_result": (C.c_int, [C.c_void_p, C.c_longlong, _P]),
    "pcas_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.c_int, _P]),
    "pcas_batch_solve": (C.c_int, [C.c_void_p, _D, _D, _D, C.POINTER(Stats), _P]),
    "pcas_batch_destroy": (C.c_int, [C.c_void_p]),
    "pcas_autotune": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.POINTER(Vol), C.POINTER(CB), C.POINTER(Params),
                                _D, _P, _P, C.c_size_t, _P, _P]),
    "pcas_tuning_get": (C.c_int, [C.POINTER(Vol), C.POINTER(CB), C.c_int, C.c_int, _P]),
    "pcas_tuning_set": (C.c_int, [C.POINTER(Vol), C.POINTER(CB), C.c_int, C.c_int, _P]),
    "pcas_tuning_clear": (C.c_int, []),
    "pcas_profile": (C.c_int, [C.c_int]),
    "pcas_profile_read": (C.c_int, [C.c_int, C.POINTER(C.c_longlong), _D]),
}

# kernel classes of pcas_profile_read (include/pcasolve.h)
KERNELS = ["warp_pca", "drr_solver", "resid", "adjoint_grad", "drr_forward", "drr_adjoint",
           "pca_dvf", "warp_volume", "localize", "init", "warp_batch", "drr_batch", "grad_f0", "graph",
           "siddon"]


def lib():
    """Load libpcasolve.so (built in-tree by ``paper_1102_1712_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_1102_1712_gb300.build.build() "
                    "(or __graft_entry__.build()); there is no fallback path")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().pcas_last_error().decode(errors="replace")


def _check(rc, allow=(OK,)):
    if rc not in allow:
        raise PcasError(rc, last_error())
    return rc


# ------------------------------------------------------------ marshalling
def vol_struct(v) -> Vol:
    if isinstance(v, Vol):
        return v
    return Vol(v["nx"], v["ny"], v["nz"], v["sx"], v["sy"], v["sz"], v["ox"], v["oy"], v["oz"])


def cb_struct(g) -> CB:
    if isinstance(g, CB):
        return g
    return CB(g["sad"], g["sdd"], g["nu"], g["nv"], g["du"], g["dv"], g.get("off_u", 0.0),
              g.get("off_v", 0.0), g["angle"])


def params_struct(p) -> Params:
    if isinstance(p, Params):
        return p
    return Params(p["mu0"], p["alpha"], p["beta"], p["mu_min"], int(p["max_iter"]),
                  int(p["max_trials"]), p["step"])


def _dev(t, name, numel=None, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL); float32 unless
    ``dtype`` (a torch dtype) says otherwise."""
    if t is None:
        return None
    import torch
    dtype = dtype or torch.float32
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _host_d(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _nvox(vol):
    v = vol_struct(vol)
    return v.nx * v.ny * v.nz


def _K(U, vol):
    N = _nvox(vol)
    if U.numel() % (3 * N):
        raise ValueError("U must hold K x 3 x N values")
    return U.numel() // (3 * N)


# ------------------------------------------------------------------- API
def workspace_bytes(vol, cb, K) -> int:
    return int(lib().pcas_workspace_bytes(C.byref(vol_struct(vol)), C.byref(cb_struct(cb)), int(K)))


class Workspace:
    """A 256-byte aligned device workspace for cost_grad / solve_projection."""

    def __init__(self, vol, cb, K, device=None):
        import torch
        n = workspace_bytes(vol, cb, K)
        if n == 0:
            raise ValueError("invalid volume / view / K for a workspace")
        self.buf = torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")
        base = self.buf.data_ptr()
        self.ptr = (base + 255) & ~255
        self.nbytes = n


def pca_dvf(mean, U, w, vol, out=None, stream=None):
    import torch
    N = _nvox(vol)
    K = _K(U, vol)
    wv = _host_d(w, K)
    if out is None:
        out = torch.empty(3 * N, dtype=torch.float32, device=U.device)
    _check(lib().pca_dvf(_dev(mean, "mean", 3 * N), _dev(U, "U"), K, wv.ctypes.data_as(_D),
                         C.byref(vol_struct(vol)), _dev(out, "dvf", 3 * N), _stream(stream)))
    return out


def warp_volume(f0, dvf, vol, out=None, stream=None):
    import torch
    N = _nvox(vol)
    if out is None:
        out = torch.empty(N, dtype=torch.float32, device=f0.device)
    _check(lib().warp_volume(_dev(f0, "f0", N), _dev(dvf, "dvf", 3 * N), C.byref(vol_struct(vol)),
                             _dev(out, "f", N), _stream(stream)))
    return out


def drr_forward(f, vol, cb, step, out=None, stream=None):
    import torch
    g = cb_struct(cb)
    if out is None:
        out = torch.empty(g.nu * g.nv, dtype=torch.float32, device=f.device)
    _check(lib().drr_forward(_dev(f, "f", _nvox(vol)), C.byref(vol_struct(vol)), C.byref(g),
                             float(step), _dev(out, "p", g.nu * g.nv), _stream(stream)))
    return out


def drr_siddon(f, vol, cb, out=None, stream=None):
    """Siddon's exact radiological path (Sec. II.B's simulation projector), for
    rendering measured images without the inverse crime."""
    import torch
    g = cb_struct(cb)
    if out is None:
        out = torch.empty(g.nu * g.nv, dtype=torch.float32, device=f.device)
    _check(lib().drr_siddon(_dev(f, "f", _nvox(vol)), C.byref(vol_struct(vol)), C.byref(g),
                            _dev(out, "p", g.nu * g.nv), _stream(stream)))
    return out


def drr_adjoint(img, vol, cb, step, out=None, stream=None):
    import torch
    g = cb_struct(cb)
    N = _nvox(vol)
    if out is None:
        out = torch.empty(N, dtype=torch.float32, device=img.device)
    _check(lib().drr_adjoint(_dev(img, "img", g.nu * g.nv), C.byref(vol_struct(vol)), C.byref(g),
                             float(step), _dev(out, "g", N), _stream(stream)))
    return out


def storage_type(U):
    """pcas_dtype of the motion model tensor (float32, bfloat16 or float16)."""
    import torch
    return {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}[U.dtype]


def cost_grad(f0, mean, U, w, y, vol, cb, step, ws: Workspace = None, stream=None):
    """Returns (J, dJ/dw (K,), (a, b)) at w.  f0, mean and U share one storage
    type (float32, bfloat16 or float16; float32 arithmetic either way)."""
    N = _nvox(vol)
    K = _K(U, vol)
    g = cb_struct(cb)
    ws = ws or Workspace(vol, cb, K, device=U.device)
    wv = _host_d(w, K)
    J = C.c_double()
    G = np.zeros(K)
    ab = np.zeros(2)
    dt = U.dtype
    _check(lib().cost_grad_typed(_dev(f0, "f0", N, dt), _dev(mean, "mean", 3 * N, dt), _dev(U, "U", None, dt),
                                 storage_type(U), K, wv.ctypes.data_as(_D), _dev(y, "y", g.nu * g.nv),
                                 C.byref(vol_struct(vol)), C.byref(g), float(step), C.byref(J),
                                 G.ctypes.data_as(_D), ab.ctypes.data_as(_D), ws.ptr, ws.nbytes,
                                 _stream(stream)))
    return J.value, G, (ab[0], ab[1])


class WorkspaceF0(Workspace):
    """Device workspace for cost_grad_f0."""

    def __init__(self, vol, cb, K, device=None):
        import torch
        n = int(lib().pcas_workspace_bytes_f0(C.byref(vol_struct(vol)), C.byref(cb_struct(cb)), int(K)))
        if n == 0:
            raise ValueError("invalid volume / view / K for a workspace")
        self.buf = torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")
        self.ptr = (self.buf.data_ptr() + 255) & ~255
        self.nbytes = n


def cost_grad_f0(f0, mean, U, w, y, vol, cb, step, want_grad=True, want_grad_f0=True,
                 ws: Workspace = None, out=None, stream=None):
    """Returns (J, dJ/dw (K,) or None, (a, b), dJ/df0 (N,) device tensor or None)."""
    import torch
    N = _nvox(vol)
    K = _K(U, vol)
    g = cb_struct(cb)
    ws = ws or WorkspaceF0(vol, cb, K, device=U.device)
    wv = _host_d(w, K)
    J = C.c_double()
    G = np.zeros(K) if (want_grad or want_grad_f0) else None
    ab = np.zeros(2)
    if want_grad_f0 and out is None:
        out = torch.empty(N, dtype=torch.float32, device=U.device)
    _check(lib().cost_grad_f0(_dev(f0, "f0", N), _dev(mean, "mean", 3 * N), _dev(U, "U"), K,
                              wv.ctypes.data_as(_D), _dev(y, "y", g.nu * g.nv), C.byref(vol_struct(vol)),
                              C.byref(g), float(step), C.byref(J),
                              None if G is None else G.ctypes.data_as(_D), ab.ctypes.data_as(_D),
                              _dev(out, "dJdf0", N) if want_grad_f0 else None, ws.ptr, ws.nbytes,
                              _stream(stream)))
    return J.value, G, (ab[0], ab[1]), (out if want_grad_f0 else None)


def cost_grad_static(f0, mean, U, w, y, vol, cb, step, stream=None):
    """cost_grad without a workspace, for callers that cannot allocate device
    memory: the library's fixed 16 MiB device scratch is used instead (see
    include/pcasolve.h for the size limit and the sharing rules).
    Returns (J, dJ/dw (K,), (a, b))."""
    N = _nvox(vol)
    K = _K(U, vol)
    g = cb_struct(cb)
    wv = _host_d(w, K)
    J = C.c_double()
    G = np.zeros(K)
    ab = np.zeros(2)
    _check(lib().cost_grad_static(_dev(f0, "f0", N), _dev(mean, "mean", 3 * N), _dev(U, "U"), K,
                                  wv.ctypes.data_as(_D), _dev(y, "y", g.nu * g.nv), C.byref(vol_struct(vol)),
                                  C.byref(g), float(step), C.byref(J), G.ctypes.data_as(_D),
                                  ab.ctypes.data_as(_D), _stream(stream)))
    return J.value, G, (ab[0], ab[1])


def solve_projection(f0, mean, U, y, vol, cb, w_init, params, ws: Workspace = None, stream=None):
    """Returns (w (K,), stats dict)."""
    N = _nvox(vol)
    K = _K(U, vol)
    g = cb_struct(cb)
    ws = ws or Workspace(vol, cb, K, device=U.device)
    w0 = _host_d(w_init, K)
    w_out = np.zeros(K)
    st = Stats()
    prm = params_struct(params)
    dt = U.dtype
    _check(lib().solve_projection_typed(_dev(f0, "f0", N, dt), _dev(mean, "mean", 3 * N, dt),
                                        _dev(U, "U", None, dt), storage_type(U), K,
                                        _dev(y, "y", g.nu * g.nv), C.byref(vol_struct(vol)), C.byref(g),
                                        w0.ctypes.data_as(_D), C.byref(prm), w_out.ctypes.data_as(_D),
                                        C.byref(st), ws.ptr, ws.nbytes, _stream(stream)))
    return w_out, {k: getattr(st, k) for k, _ in Stats._fields_}


def localize_tumor(mean, U, w, vol, c_ref, max_iter=50, tol_mm=1e-6, stream=None):
    """Returns (c (3,), converged)."""
    N = _nvox(vol)
    K = _K(U, vol)
    wv = _host_d(w, K)
    cr = _host_d(c_ref, 3)
    out = np.zeros(3)
    dt = U.dtype
    rc = lib().localize_tumor_typed(_dev(mean, "mean", 3 * N, dt), _dev(U, "U", None, dt), storage_type(U), K,
                                    wv.ctypes.data_as(_D), C.byref(vol_struct(vol)), cr.ctypes.data_as(_D),
                                    int(max_iter), float(tol_mm), out.ctypes.data_as(_D), _stream(stream))
    _check(rc, allow=(OK, NOT_CONVERGED))
    return out, rc == OK


def lp_fit(trace, L):
    tr = np.ascontiguousarray(trace, dtype=np.float64)
    T, K = tr.shape
    c = np.zeros((K, L))
    _check(lib().lp_fit(tr.ctypes.data_as(_D), T, K, int(L), c.ctypes.data_as(_D)))
    return c


def lp_predict(hist, c):
    """hist[l-1] = w*(t-l), shape (L, K); c shape (K, L)."""
    h = np.ascontiguousarray(hist, dtype=np.float64)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    L, K = h.shape
    w0 = np.zeros(K)
    _check(lib().lp_predict(h.ctypes.data_as(_D), cc.ctypes.data_as(_D), K, L, w0.ctypes.data_as(_D)))
    return w0


class Solver:
    """Device-driven solve of one reference CT / motion model / detector shape:
    solve_projection captured as a CUDA graph with conditional loops (see
    include/pcasolve.h).  Keeps references to the tensors it was built on."""

    def __init__(self, f0, mean, U, vol, cb, params, device=None, stream=None):
        import torch
        self.K = _K(U, vol)
        self.vol, self.cb = vol_struct(vol), cb_struct(cb)
        self.tensors = (f0, mean, U)
        N = _nvox(vol)
        dt = U.dtype
        n = int(lib().pcas_solver_workspace_bytes(C.byref(self.vol), C.byref(self.cb), self.K))
        if n == 0:
            raise ValueError("invalid volume / view / K")
        self.buf = torch.empty(n + 256, dtype=torch.uint8, device=device or U.device)
        ptr = (self.buf.data_ptr() + 255) & ~255
        h = C.c_void_p()
        _check(lib().pcas_solver_create(C.byref(h), _dev(f0, "f0", N, dt), _dev(mean, "mean", 3 * N, dt),
                                        _dev(U, "U", None, dt), storage_type(U), self.K, C.byref(self.vol),
                                        C.byref(self.cb), C.byref(params_struct(params)), ptr, n,
                                        _stream(stream)))
        self.h = h

    def y_buffer(self):
        """Device address of the solver's own image buffer (nu * nv float32)."""
        return lib().pcas_solver_y_buffer(self.h)

    def solve(self, y, w_init, angle=None, off_u=None, off_v=None, stream=None):
        """Returns (w (K,), stats dict).  y: CUDA float32 tensor or None (use y_buffer())."""
        nu, nv = self.cb.nu, self.cb.nv
        w0 = _host_d(w_init, self.K)
        w_out = np.zeros(self.K)
        st = Stats()
        _check(lib().pcas_solver_solve(self.h, None if y is None else _dev(y, "y", nu * nv),
                                       float(self.cb.angle_rad if angle is None else angle),
                                       float(self.cb.off_u if off_u is None else off_u),
                                       float(self.cb.off_v if off_v is None else off_v),
                                       w0.ctypes.data_as(_D), w_out.ctypes.data_as(_D), C.byref(st),
                                       _stream(stream)))
        return w_out, {k: getattr(st, k) for k, _ in Stats._fields_}

    # ---- fixed-angle fluoroscopy (Sec. IV): the constant part of P^T cached
    def fixed_view_bytes(self, angle, stream=None):
        """Device bytes of the fixed-view cache of P^T at this gantry angle."""
        n = int(lib().pcas_solver_fixed_view_bytes(self.h, float(angle), _stream(stream)))
        if n == 0:
            raise ValueError("no fixed-view cache for this solver and angle: " + last_error())
        return n

    def fix_view(self, angle, stream=None):
        """Builds the fixed-view cache for solves at exactly this angle (device
        memory held by the solver object); angle None turns it off."""
        import torch
        if angle is None:
            _check(lib().pcas_solver_fix_view(self.h, 0.0, None, 0, _stream(stream)))
            self.pt_buf = None
            return 0
        n = self.fixed_view_bytes(angle, stream)
        buf = torch.empty(n + 256, dtype=torch.uint8, device=self.buf.device)
        ptr = (buf.data_ptr() + 255) & ~255
        _check(lib().pcas_solver_fix_view(self.h, float(angle), ptr, n, _stream(stream)))
        self.pt_buf = buf
        return n

    # ---- runs of consecutive projections (warm start and localisation on the device)
    def seq_begin(self, lp_coef, c_ref, loc_max_iter=50, loc_tol_mm=1e-6, w_hist=None, stream=None):
        """Starts a run.  lp_coef: (K, L) Eq. (3) coefficients (lp_fit); c_ref:
        tumour centroid of the reference CT (mm); w_hist: (n, K) solutions
        before the run, latest first (or None)."""
        c = np.ascontiguousarray(lp_coef, dtype=np.float64)
        if c.ndim != 2 or c.shape[0] != self.K:
            raise ValueError(f"lp_coef must be (K={self.K}, L)")
        cr = _host_d(c_ref, 3)
        if w_hist is None or len(w_hist) == 0:
            h, n = None, 0
        else:
            h = np.ascontiguousarray(w_hist, dtype=np.float64).reshape(-1, self.K)
            n = h.shape[0]
        _check(lib().pcas_solver_seq_begin(self.h, c.ctypes.data_as(_D), c.shape[1], cr.ctypes.data_as(_D),
                                           int(loc_max_iter), float(loc_tol_mm),
                                           None if h is None else h.ctypes.data_as(_D), n, _stream(stream)))

    def seq_enqueue(self, y, angle, w_first=None, stream=None):
        """Queues one projection (y: float32 tensor on the device or in pinned
        host memory); returns its ticket without waiting."""
        nu, nv = self.cb.nu, self.cb.nv
        if y is None or not y.is_contiguous() or y.numel() != nu * nv or str(y.dtype) != "torch.float32":
            raise ValueError(f"y must be a contiguous float32 tensor of {nu * nv} values")
        if not (y.is_cuda or y.is_pinned()):
            raise ValueError("y must live on the device or in pinned host memory")
        wf = None if w_first is None else _host_d(w_first, self.K)
        t = C.c_longlong()
        _check(lib().pcas_solver_seq_enqueue(self.h, y.data_ptr(), float(angle),
                                             None if wf is None else wf.ctypes.data_as(_D), C.byref(t),
                                             _stream(stream)))
        return t.value

    def seq_result(self, ticket):
        """Waits for a queued projection; returns (w (K,), stats dict, c (3,), converged)."""
        r = SeqResult()
        _check(lib().pcas_solver_seq_result(self.h, int(ticket), C.byref(r)))
        stats = {k: getattr(r.stats, k) for k, _ in Stats._fields_}
        return np.array(r.w[:self.K]), stats, np.array(r.c[:]), bool(r.loc_converged)

    def solve_sequence(self, ys, angles, w_first=None, lookahead=32, stream=None):
        """Queues every projection of ys (indexable, one tensor per angle) in
        the current run, keeping at most ``lookahead`` in flight; returns the
        list of seq_result tuples in order."""
        lookahead = max(1, min(int(lookahead), 48))
        tickets, out = [], []
        for t in range(len(angles)):
            tickets.append(self.seq_enqueue(ys[t], angles[t], w_first, stream))
            if len(tickets) - len(out) >= lookahead:
                out.append(self.seq_result(tickets[len(out)]))
        while len(out) < len(tickets):
            out.append(self.seq_result(tickets[len(out)]))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().pcas_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many device-driven solves (uneven sizes) as branches of one CUDA graph:
    one launch solves them all.  ys[i]: CUDA tensor copied into solver i's image
    buffer at each launch (or None)."""

    def __init__(self, solvers, ys=None, stream=None):
        self.solvers = list(solvers)
        n = len(self.solvers)
        arr = (C.c_void_p * n)(*[s.h.value for s in self.solvers])
        ysrc = None
        if ys is not None:
            self.ys = list(ys)
            ysrc = (C.c_void_p * n)(*[None if y is None else _dev(y, "y") for y in self.ys])
        h = C.c_void_p()
        _check(lib().pcas_batch_create(C.byref(h), arr, ysrc, n, _stream(stream)))
        self.h = h

    def solve(self, angles, w_init, stream=None):
        """angles (n,), w_init list of n K_i-vectors -> (list of w, list of stats dicts)."""
        n = len(self.solvers)
        W0 = np.zeros((n, KMAX))
        for i, w in enumerate(w_init):
            W0[i, :len(w)] = w
        ang = _host_d(angles, n)
        Wout = np.zeros((n, KMAX))
        st = (Stats * n)()
        _check(lib().pcas_batch_solve(self.h, ang.ctypes.data_as(_D), W0.ctypes.data_as(_D),
                                      Wout.ctypes.data_as(_D), st, _stream(stream)))
        return ([Wout[i, :s.K].copy() for i, s in enumerate(self.solvers)],
                [{k: getattr(st[i], k) for k, _ in Stats._fields_} for i in range(n)])

    def close(self):
        if getattr(self, "h", None):
            lib().pcas_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tuning(C.Structure):
    """pcas_tuning: launch shapes of one size bucket (include/pcasolve.h)."""
    _fields_ = [("ray_lw1", C.c_int), ("chunk1", C.c_int), ("voxel_tile", C.c_int), ("gather_per_sm", C.c_int),
                ("skip_empty", C.c_int),
                ("ray_lw4", C.c_ubyte * 8), ("chunk", C.c_ubyte * 8), ("swap", C.c_ubyte * 8)]
    SCALARS = ("ray_lw1", "chunk1", "voxel_tile", "gather_per_sm", "skip_empty")
    OPTIONAL = {"skip_empty": 1}      # entries written before the field existed
    PER_BIN = ("ray_lw4", "chunk", "swap")

    def as_dict(self):
        d = {k: getattr(self, k) for k in self.SCALARS}
        d.update({k: list(getattr(self, k)) for k in self.PER_BIN})
        return d


def _tuning_struct(d):
    t = Tuning()
    for k in Tuning.SCALARS:
        setattr(t, k, int(d[k] if k in d else Tuning.OPTIONAL[k]))
    for k in Tuning.PER_BIN:
        arr = getattr(t, k)
        vals = d[k] if hasattr(d[k], "__len__") else [d[k]] * 8
        for b, v in enumerate(vals):
            arr[b] = int(v)
    return t


def autotune(f0, mean, U, y, vol, cb, params, w_init=None, ws: Workspace = None, stream=None):
    """Measure launch shapes on this problem and store the fastest for its size
    bucket (synchronous, about 130 short trial solves).  Returns the entry."""
    K = _K(U, vol)
    N = _nvox(vol)
    dt = U.dtype
    g = cb_struct(cb)
    ws = ws or Workspace(vol, cb, K, device=U.device)
    w0 = None if w_init is None else _host_d(w_init, K)
    out = Tuning()
    _check(lib().pcas_autotune(_dev(f0, "f0", N, dt), _dev(mean, "mean", 3 * N, dt), _dev(U, "U", None, dt),
                               storage_type(U), K, C.byref(vol_struct(vol)), C.byref(g),
                               C.byref(params_struct(params)), None if w0 is None else w0.ctypes.data_as(_D),
                               _dev(y, "y", g.nu * g.nv), ws.ptr, ws.nbytes, C.byref(out), _stream(stream)))
    return out.as_dict()


def tuning_get(vol, cb, K, dtype=None):
    """The launch shapes in force for this problem's size bucket."""
    out = Tuning()
    _check(lib().pcas_tuning_get(C.byref(vol_struct(vol)), C.byref(cb_struct(cb)), int(K),
                                 F32 if dtype is None else int(dtype), C.byref(out)))
    return out.as_dict()


def tuning_set(vol, cb, K, tuning, dtype=None):
    _check(lib().pcas_tuning_set(C.byref(vol_struct(vol)), C.byref(cb_struct(cb)), int(K),
                                 F32 if dtype is None else int(dtype), C.byref(_tuning_struct(tuning))))


def tuning_clear():
    _check(lib().pcas_tuning_clear())


def profile(on: bool):
    """Reset the per-kernel launch counters; time every launch with CUDA events while on."""
    _check(lib().pcas_profile(1 if on else 0))


def profile_read():
    """{kernel class: (launches, summed event ms)} since the last profile() reset."""
    out = {}
    for i, name in enumerate(KERNELS):
        n = C.c_longlong()
        ms = C.c_double()
        _check(lib().pcas_profile_read(i, C.byref(n), C.byref(ms)))
        out[name] = (int(n.value), float(ms.value))
    return out


def default_params(step_mm, **kw):
    """Appendix constants scaled for O(1) coefficients (mu0 2 -> 0.2, mu_min 0.1 -> 0.01)."""
    d = dict(mu0=0.2, alpha=0.1, beta=0.5, mu_min=0.01, max_iter=10, max_trials=30, step=float(step_mm))
    d.update(kw)
    return d
