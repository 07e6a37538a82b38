"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *generates inputs*: volumes, phantoms, eigenvector fields,
breathing traces, gantry angles and noise.  It holds none of the method's
arithmetic (no DVF synthesis, warp, projection, cost or solve), so both the
CUDA path and the oracle can draw from it without sharing any of the method.

The datasets of the paper (NCAT digital phantom, RPM breathing trace,
physical phantom and patient 4DCT/CBCT, Sec. II.B-II.D) are not available;
these generators stand in for them:

* ``phantom``: body ellipsoid 0.02/mm, two lung ellipsoids 0.005/mm and a
  spherical tumour 0.02/mm inside the right lung, voxel value = analytic value
  at the voxel centre (Sec. II.B uses an anatomical phantom of this kind).
* ``eigen_dvfs``: K smooth random fields (N(0,1) per component, Gaussian
  smoothing sigma = 8 mm with zero boundary) scaled so that u_1's largest |SI|
  entry is 10 mm and every other u_k's dominant component peaks at 10 mm;
  with the mean field zero, w = 1 moves the peak voxel 10 mm (Sec. II.A keeps
  three eigenvectors).
* ``breathing_trace``: w_1(t) = (A / 10 mm) * (1 - cos(2 pi t / T)) / 2 from
  end-of-exhale (the reference phase, w = 0) to end-of-inhale, w_2 = 0.3 w_1
  lagging T/8 and w_3 = 0.15 w_1 leading T/8 (hysteresis); the irregular form
  jitters each cycle's period and amplitude by U(-30 %, +30 %) and adds a
  linear baseline drift (Sec. II.B, Table 1).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "volume", "cone_beam", "phantom", "eigen_dvfs", "translation_dvfs", "breathing_trace",
    "gantry_angles", "gaussian_noise", "rng",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed)))


def volume(nx: int, ny: int, nz: int, sx: float, sy: float, sz: float) -> dict:
    """Grid centred on the isocentre: voxel (0,0,0) at o = -(n-1) s / 2."""
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), sx=float(sx), sy=float(sy), sz=float(sz),
                ox=-0.5 * (nx - 1) * sx, oy=-0.5 * (ny - 1) * sy, oz=-0.5 * (nz - 1) * sz)


def cone_beam(nu: int, nv: int, du: float, dv: float, angle_rad: float = 0.0,
              sad: float = 1000.0, sdd: float = 1500.0, off_u: float = 0.0,
              off_v: float = 0.0) -> dict:
    return dict(sad=float(sad), sdd=float(sdd), nu=int(nu), nv=int(nv), du=float(du),
                dv=float(dv), off_u=float(off_u), off_v=float(off_v), angle=float(angle_rad))


def _centres(vol: dict):
    x = vol["ox"] + vol["sx"] * np.arange(vol["nx"])
    y = vol["oy"] + vol["sy"] * np.arange(vol["ny"])
    z = vol["oz"] + vol["sz"] * np.arange(vol["nz"])
    return x, y, z


def _ellipsoid_mask(vol, c, ax):
    x, y, z = _centres(vol)
    X = ((x - c[0]) / ax[0]) ** 2
    Y = ((y - c[1]) / ax[1]) ** 2
    Z = ((z - c[2]) / ax[2]) ** 2
    return (Z[:, None, None] + Y[None, :, None] + X[None, None, :]) <= 1.0


def phantom(vol: dict, tumor_radius_mm: float, seed: int,
            mu_body: float = 0.02, mu_lung: float = 0.005, mu_tumor: float = 0.02):
    """Ellipsoid chest phantom.  Returns (f0 float32 [nz,ny,nx], tumour centre (3,) mm)."""
    g = rng(seed)
    ext = np.array([vol["nx"] * vol["sx"], vol["ny"] * vol["sy"], vol["nz"] * vol["sz"]])
    jit = lambda n, s: 1.0 + s * g.uniform(-1.0, 1.0, n)  # noqa: E731
    body_ax = np.array([0.44, 0.34, 0.62]) * ext * jit(3, 0.03)
    body_c = 0.01 * ext * g.uniform(-1, 1, 3)
    lung_ax = np.array([0.14, 0.2, 0.38]) * ext
    lungs = []
    for side in (+1.0, -1.0):
        c = np.array([side * 0.2 * ext[0], 0.02 * ext[1], 0.05 * ext[2]]) + 0.01 * ext * g.uniform(-1, 1, 3)
        lungs.append((c, lung_ax * jit(3, 0.05)))
    f0 = np.zeros((vol["nz"], vol["ny"], vol["nx"]), np.float32)
    f0[_ellipsoid_mask(vol, body_c, body_ax)] = mu_body
    for c, ax in lungs:
        f0[_ellipsoid_mask(vol, c, ax)] = mu_lung
    # tumour inside the right lung, away from its wall
    c_lung, ax_lung = lungs[0]
    room = np.maximum(ax_lung - 1.5 * tumor_radius_mm, 0.0)
    c_t = c_lung + 0.3 * room * g.uniform(-1, 1, 3)
    f0[_ellipsoid_mask(vol, c_t, np.full(3, float(tumor_radius_mm)))] = mu_tumor
    return f0, c_t.astype(np.float64)


def _smooth(a: np.ndarray, sig_vox) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma=sig_vox, mode="constant", cval=0.0, truncate=3.0)


def _upsample_linear(a: np.ndarray, shape) -> np.ndarray:
    """Separable linear interpolation of a coarse grid onto ``shape`` (end points aligned)."""
    out = a.astype(np.float32)
    for ax, n in enumerate(shape):
        m = out.shape[ax]
        if m == n:
            continue
        x = np.linspace(0.0, m - 1.0, n, dtype=np.float64)
        i0 = np.minimum(np.floor(x).astype(np.int64), m - 2)
        t = (x - i0).astype(np.float32)
        sh = [1] * out.ndim
        sh[ax] = n
        t = t.reshape(sh)
        out = np.take(out, i0, axis=ax) * (1 - t) + np.take(out, i0 + 1, axis=ax) * t
    return out


def eigen_dvfs(vol: dict, K: int, seed: int, sigma_mm: float = 8.0, peak_mm: float = 10.0,
               dtype=np.float32, coarse=(1, 1, 1)) -> np.ndarray:
    """K smoothed random vector fields, shape [K, 3, nz*ny*nx], in mm.

    ``coarse`` = (cz, cy, cx) > 1 draws the white noise on a grid that much
    coarser, smooths it there (same sigma in mm) and interpolates linearly to
    the full grid: for large volumes, where smoothing at full resolution would
    take minutes.  The fields stay smooth at the sigma scale."""
    g = rng(seed)
    shape = (vol["nz"], vol["ny"], vol["nx"])
    cz, cy, cx = coarse
    cshape = (-(-shape[0] // cz), -(-shape[1] // cy), -(-shape[2] // cx))
    sig = (sigma_mm / (vol["sz"] * cz), sigma_mm / (vol["sy"] * cy), sigma_mm / (vol["sx"] * cx))
    N = int(np.prod(shape))
    U = np.empty((K, 3, N), dtype)

    def field():
        f = _smooth(g.standard_normal(cshape), sig)
        return f if cshape == shape else _upsample_linear(f, shape)

    for k in range(K):
        comps = [field() for _ in range(3)]
        peaks = [np.abs(c).max() for c in comps]
        ref = peaks[2] if k == 0 else max(peaks)
        for c in range(3):
            U[k, c] = (comps[c] * (peak_mm / ref)).ravel().astype(dtype)
    return U


def translation_dvfs(vol: dict, K: int = 3, mm: float = 10.0, dtype=np.float32) -> np.ndarray:
    """u_k = constant unit vector e_k times ``mm`` (K <= 3): x = U w is a rigid shift."""
    N = vol["nx"] * vol["ny"] * vol["nz"]
    U = np.zeros((K, 3, N), dtype)
    for k in range(K):
        U[k, k] = mm
    return U


def breathing_trace(n: int, fps: float, period_s: float = 4.0, amp_mm: float = 15.0,
                    K: int = 3, irregular: bool = False, drift_mm: float = 0.0,
                    jitter: float = 0.3, seed: int = 0, t0: float = 0.0,
                    amp_jitter: float | None = None) -> np.ndarray:
    """Planted coefficients w(t), shape [n, K], sampled at ``fps``.  Irregular
    traces scale each cycle's period by 1 + U(-jitter, jitter) and its
    amplitude by 1 + U(-amp_jitter, amp_jitter) (amp_jitter defaults to jitter)."""
    amp_jitter = jitter if amp_jitter is None else amp_jitter
    g = rng(seed)
    t = t0 + np.arange(n) / fps
    tmax = t[-1] + 2 * period_s
    # cycle boundaries with per-cycle period/amplitude factors
    starts, periods, amps = [t0 - period_s], [], []
    while starts[-1] < tmax:
        pf = 1.0 + (g.uniform(-jitter, jitter) if irregular else 0.0)
        af = 1.0 + (g.uniform(-amp_jitter, amp_jitter) if irregular else 0.0)
        periods.append(period_s * pf)
        amps.append(amp_mm * af)
        starts.append(starts[-1] + periods[-1])
    starts = np.array(starts[:-1])
    periods, amps = np.array(periods), np.array(amps)

    def phase_amp(tt):
        idx = np.clip(np.searchsorted(starts, tt, side="right") - 1, 0, len(starts) - 1)
        return (tt - starts[idx]) / periods[idx], amps[idx], periods[idx]

    W = np.zeros((n, K))
    lags = [0.0, -0.125, 0.125]
    scale = [1.0, 0.3, 0.15]
    for k in range(min(K, 3)):
        ph, A, _ = phase_amp(t + lags[k] * period_s)
        W[:, k] = scale[k] * (A / 10.0) * 0.5 * (1.0 - np.cos(2 * math.pi * ph))
    for k in range(3, K):
        ph, A, _ = phase_amp(t + 0.25 * period_s)
        W[:, k] = 0.05 * (A / 10.0) * np.sin(2 * math.pi * ph)
    if drift_mm:
        W[:, 0] += (drift_mm / 10.0) * (t - t0) / max(t[-1] - t0, 1e-9)
    return W


def gantry_angles(n: int, total_deg: float = 360.0, start_deg: float = 0.0) -> np.ndarray:
    return np.deg2rad(start_deg + total_deg * np.arange(n) / n)


def gaussian_noise(shape, sigma: float, seed: int, dtype=np.float32) -> np.ndarray:
    return (sigma * rng(seed).standard_normal(shape)).astype(dtype)
