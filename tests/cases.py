"""Seeded test problems shared by the GPU parity tests.  Inputs come from the
generators in ``paper_1102_1712_gb300.synth``; the measured projection y is
rendered by the oracle (never by the CUDA path)."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1102_1712_gb300 import synth as S

# The tiny workload: 64x64x32 CT at 4 mm, K = 3, 128x96 detector at 3.1 mm,
# gantry 0 deg, planted w = (1.2, -0.4, 0.3), 1 % noise, 20 iterations from 0.
TINY = dict(vol=(64, 64, 32, 4.0, 4.0, 4.0), tumor=15.0, K=3, det=(128, 96, 3.1, 3.1),
            angle=0.0, w_true=(1.2, -0.4, 0.3), noise=0.01, seeds=(1, 2, 3), iters=20)

# The paper-shaped sequence workload: 256x256x100 CT at 2x2x2.5 mm, K = 3,
# 512x384 detector at 0.776 mm, 600 views over 360 deg at 10 fps.
SEQUENCE = dict(vol=(256, 256, 100, 2.0, 2.0, 2.5), tumor=20.0, K=3, det=(512, 384, 0.776, 0.776),
                n_proj=600, fps=10.0, period=4.0, amp=15.0, seeds=(10, 11, 12))


def make_problem(vol_dims, K, det, angle, w_true, noise=0.01, seeds=(1, 2, 3), tumor=15.0,
                 off=(0.0, 0.0), with_mean=False, step=None, scale_ab=None):
    vol = S.volume(*vol_dims)
    cb = S.cone_beam(det[0], det[1], det[2], det[3], angle, off_u=off[0], off_v=off[1])
    step = step if step is not None else 0.5 * min(vol["sx"], vol["sy"], vol["sz"])
    f0, c_ref = S.phantom(vol, tumor, seed=seeds[0])
    U = S.eigen_dvfs(vol, K, seed=seeds[1])
    N = f0.size
    mean = None
    if with_mean:
        mean = (0.3 * S.eigen_dvfs(vol, 1, seed=seeds[1] + 100)[0]).astype(np.float32)
    w_true = np.asarray(w_true, float)
    y = O.drr_forward(O.warp_volume(f0, O.pca_dvf(mean, U, w_true, vol), vol), vol, cb, step)
    if scale_ab is not None:
        y = (y - scale_ab[1]) / scale_ab[0]
    if noise:
        y = y + S.gaussian_noise(y.shape, noise * np.abs(y).max(), seed=seeds[2], dtype=np.float64)
    return dict(vol=vol, cb=cb, step=step, f0=f0, U=U, mean=mean, c_ref=c_ref, w_true=w_true,
                y=y.astype(np.float32), N=N, K=K)


def tiny_problem():
    t = TINY
    return make_problem(t["vol"], t["K"], t["det"], t["angle"], t["w_true"], t["noise"], t["seeds"],
                        t["tumor"])


def to_dev(pb, dev="cuda"):
    import torch
    d = dict(f0=torch.from_numpy(pb["f0"].ravel()).to(dev), U=torch.from_numpy(pb["U"].ravel()).to(dev),
             y=torch.from_numpy(pb["y"]).to(dev))
    d["mean"] = None if pb["mean"] is None else torch.from_numpy(pb["mean"].ravel()).to(dev)
    return d
