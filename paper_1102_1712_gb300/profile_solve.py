"""Runs a few solves of one synthetic problem, for profiler captures.

    python -m paper_1102_1712_gb300.profile_solve --angle-deg 45 --solves 3 \\
        [--tuning '{"ray_lw1": 3, ...}'] [--vol nx,ny,nz,sx,sy,sz] [--det nu,nv,pixel_mm] [--K 3]

Defaults: the 256x256x100 (2x2x2.5 mm) sequence volume, K = 3, a 512x384
detector at 0.776 mm, seeded phantom and eigenvector fields, the measured
image rendered by Siddon's projector at w = (1, 0.3, 0.15), each solve started
from 0.8 w.  With --tuning the launch shapes of the bucket are set first (else
the defaults), so a capture sees the same kernels as a tuned run.  Every
solve is the host-driven solve_projection (one launch per kernel).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--vol", default="256,256,100,2.0,2.0,2.5")
    ap.add_argument("--det", default="512,384,0.776")
    ap.add_argument("--K", type=int, default=3)
    ap.add_argument("--angle-deg", type=float, default=45.0)
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--tuning", default=None, help="pcas_tuning entry as JSON")
    a = ap.parse_args(argv)
    import torch

    from . import build as B
    from . import pcasolve as P
    from . import synth as S

    B.build()
    v = [float(x) for x in a.vol.split(",")]
    d = [float(x) for x in a.det.split(",")]
    vol = S.volume(int(v[0]), int(v[1]), int(v[2]), v[3], v[4], v[5])
    cb = S.cone_beam(int(d[0]), int(d[1]), d[2], d[2], np.deg2rad(a.angle_deg))
    step = 0.5 * min(v[3:])
    f0, _ = S.phantom(vol, 20.0, seed=10)
    coarse = (1, 1, 1) if vol["nx"] * vol["ny"] * vol["nz"] <= 8_000_000 else (2, 2, 2)
    U = S.eigen_dvfs(vol, a.K, seed=11, coarse=coarse)
    tf0, tU = torch.from_numpy(f0.ravel()).cuda(), torch.from_numpy(U.ravel()).cuda()
    w_true = np.array([1.0, 0.3, 0.15] + [0.0] * max(0, a.K - 3))[:a.K]
    y = P.drr_siddon(P.warp_volume(tf0, P.pca_dvf(None, tU, w_true, vol), vol), vol, cb)
    if a.tuning:
        P.tuning_set(vol, cb, a.K, json.loads(a.tuning))
    prm = P.default_params(step)
    ws = P.Workspace(vol, cb, a.K)
    for _ in range(a.solves):
        w, st = P.solve_projection(tf0, None, tU, y, vol, cb, 0.8 * w_true, prm, ws=ws)
    torch.cuda.synchronize()
    print(json.dumps({"tuning": P.tuning_get(vol, cb, a.K), "w": w.tolist(), "stats": st}))


if __name__ == "__main__":
    main()
