"""Benchmark: projections/s of the single-projection PCA motion solve on the
paper-shaped sequence workload (256x256x100 CT at 2x2x2.5 mm, K = 3, 512x384
detector at 0.776 mm, 600 views over 360 deg at 10 fps, sinusoidal 4 s / 15 mm
breathing), one step = one projection: linear-prediction warm start (Eq. 3),
the alternating solve of the Appendix (warp + DRR + adjoint iterations with
Armijo backtracking) and tumour localisation (Sec. II.A).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores over a bounded sample of the same workload.
Inputs are synthetic (seeded phantom, eigenvector fields and breathing trace);
the measured projections are rendered on the GPU by this library's own warp
and projector at the planted coefficients plus 1 % Gaussian noise.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="sequence-256x256x100-K3-512x384", vol=(256, 256, 100, 2.0, 2.0, 2.5), K=3,
                det=(512, 384, 0.776, 0.776), n_proj=600, fps=10.0, period_s=4.0, amp_mm=15.0,
                tumor_mm=20.0, seeds=dict(phantom=10, dvf=11, noise=12), noise=0.01)
METRIC = "projections/s solved (warp+DRR+adjoint iters), % HBM roofline, mm error"

# Batch workload (not the default bench line): 64 independent solves, volumes
# 128^2x64 / 192^2x96 / 256^2x128 (500 mm in-plane, 250 mm axial field of
# view), K 3 / 5, detectors 256x192 ... 1024x768 with 400 mm / nu pixels,
# gantry angles U[0, 360), planted w ~ N(0, 1), each solve from w = 0.
BATCH = dict(name="batch-64-uneven", n=64, sizes=((128, 128, 64), (192, 192, 96), (256, 256, 128)), Ks=(3, 5),
             dets=((256, 192), (512, 384), (768, 576), (1024, 768)), fov=(500.0, 250.0), noise=0.01)

# Precision workload (not the default bench line): 512x512x160 CT at 1x1x2 mm,
# K = 5, 1024x768 detector at 0.388 mm, 300 views, irregular trace (period
# 3-6 s, amplitude 8-20 mm, 5 mm drift); model and CT stored in float32,
# bfloat16 and float16 in turn.
PRECISION = dict(name="precision-512x512x160-K5-1024x768", vol=(512, 512, 160, 1.0, 1.0, 2.0), K=5,
                 det=(1024, 768, 0.388, 0.388), n_proj=300, fps=10.0, period_s=4.5, amp_mm=14.0,
                 jitter=1.0 / 3.0, amp_jitter=3.0 / 7.0, drift_mm=5.0, tumor_mm=20.0,
                 seeds=dict(phantom=30, dvf=31, noise=32, trace=33), noise=0.01)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--irregular", action="store_true", help="irregular breathing trace")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="sequence",
                    choices=["sequence", "fluoro", "precision", "batch", "oracle"],
                    help="sequence: the default line; fluoro: the same sequence at one fixed gantry angle "
                         "(fluoroscopy); precision: float32 vs bfloat16 vs float16 storage; "
                         "batch: 64 uneven solves in one graph launch vs one after another; "
                         "oracle: the FP64 oracle's timings on the host cores (no GPU work)")
    ap.add_argument("--projector", default="siddon", choices=["siddon", "trilinear"],
                    help="renderer of the measured images: Siddon's exact path (Sec. II.B, no inverse "
                         "crime) or the solver's own trilinear projector")
    ap.add_argument("--angle-deg", type=float, default=90.0, help="gantry angle of the fluoro workload")
    ap.add_argument("--no-extra", action="store_true",
                    help="sequence workload: leave out the short batch and precision sub-objects")
    ap.add_argument("--no-view-cache", action="store_true",
                    help="fluoro workload: compute P^T's weights in every gradient instead of caching them")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of tuning the size bucket first")
    ap.add_argument("--tuning", default=None,
                    help="launch shapes of the sequence bucket as JSON (pcas_tuning), instead of tuning")
    return ap.parse_args()


def max_over_ranks(values, ws_, device):
    """Elementwise maximum of per-rank timings over all ranks (identity on one)."""
    if ws_ <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def replica_throughput(ws_, steps, t_max_s):
    """Whole-job projections/s of N independent replicas (weak scaling): every
    rank solves `steps` projections, the job lasts as long as the slowest rank."""
    return ws_ * steps / t_max_s


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- inputs
def workload_name(args):
    base = WORKLOAD["name"] + ("-irregular" if args.irregular else "-regular")
    if args.workload == "fluoro":
        base = base.replace("sequence", "fluoro") + f"-{args.angle_deg:g}deg"
    return base + ("-siddon" if args.projector == "siddon" else "-trilinear")


def fixed_angles(args, angles):
    """The fluoro workload projects every frame at one gantry angle."""
    return np.full_like(angles, np.deg2rad(args.angle_deg)) if args.workload == "fluoro" else angles


def make_inputs(irregular: bool):
    from paper_1102_1712_gb300 import synth as S
    W = WORKLOAD
    vol = S.volume(*W["vol"])
    f0, c_ref = S.phantom(vol, W["tumor_mm"], seed=W["seeds"]["phantom"])
    U = S.eigen_dvfs(vol, W["K"], seed=W["seeds"]["dvf"])
    if irregular:
        trace = S.breathing_trace(W["n_proj"], W["fps"], W["period_s"], W["amp_mm"], K=W["K"],
                                  irregular=True, drift_mm=3.0, seed=13)
    else:
        trace = S.breathing_trace(W["n_proj"], W["fps"], W["period_s"], W["amp_mm"], K=W["K"])
    # prediction model fitted on the regular training trace at the projection rate (Sec. II.A)
    train = S.breathing_trace(400, W["fps"], W["period_s"], W["amp_mm"], K=W["K"], t0=0.37)
    angles = S.gantry_angles(W["n_proj"], 360.0)
    return vol, f0, c_ref, U, trace, train, angles


def precision_inputs():
    """The precision workload's inputs (numpy): 512x512x160 phantom at 1x1x2 mm,
    K = 5 eigenvector fields smoothed on a coarse grid, the irregular trace, the
    training trace of the predictor and the gantry angles."""
    from paper_1102_1712_gb300 import synth as S
    W = PRECISION
    vol = S.volume(*W["vol"])
    f0, c_ref = S.phantom(vol, W["tumor_mm"], seed=W["seeds"]["phantom"])
    U = S.eigen_dvfs(vol, W["K"], seed=W["seeds"]["dvf"], coarse=(2, 4, 4))
    trace = S.breathing_trace(W["n_proj"], W["fps"], W["period_s"], W["amp_mm"], K=W["K"], irregular=True,
                              drift_mm=W["drift_mm"], jitter=W["jitter"], amp_jitter=W["amp_jitter"],
                              seed=W["seeds"]["trace"])
    train = S.breathing_trace(400, W["fps"], W["period_s"], W["amp_mm"], K=W["K"], t0=0.37)
    angles = S.gantry_angles(W["n_proj"], 360.0)
    return vol, f0, c_ref, U, trace, train, angles


def batch_inputs():
    """The batch workload's 64 problems (numpy): volume, K, view, phantom,
    eigenvector fields (one array per (size, K) model, shared), tumour centre,
    planted w and ray-march step."""
    from paper_1102_1712_gb300 import synth as S
    W = BATCH
    g = S.rng(99)
    models = {}
    probs = []
    for i in range(W["n"]):
        nx, ny, nz = W["sizes"][i % 3]
        K = W["Ks"][i % 2]
        nu, nv = W["dets"][i % 4]
        vol = S.volume(nx, ny, nz, W["fov"][0] / nx, W["fov"][0] / ny, W["fov"][1] / nz)
        key = (i % 3, K)
        if key not in models:
            coarse = (1, 1, 1) if nx <= 128 else (2, 2, 2)
            models[key] = S.eigen_dvfs(vol, K, seed=200 + 10 * (i % 3) + K, coarse=coarse)
        f0, c_ref = S.phantom(vol, 15.0, seed=100 + i)
        cb = S.cone_beam(nu, nv, 400.0 / nu, 400.0 / nu, float(g.uniform(0, 2 * np.pi)))
        w_true = g.standard_normal(K)
        probs.append(dict(vol=vol, K=K, cb=cb, f0=f0, U=models[key], model=key, c_ref=c_ref, w_true=w_true,
                          step=0.5 * min(vol["sx"], vol["sy"], vol["sz"])))
    return probs


def batch_fingerprint_parts(probs):
    """What input_fingerprint hashes for the batch workload: the planted w and
    tumour centres of the 64 problems, and samples of every model and phantom."""
    seen, parts = set(), []
    for pb in probs:
        if pb["model"] not in seen:
            seen.add(pb["model"])
            parts.append(np.asarray(pb["U"]).ravel()[::97])
        parts.append(np.asarray(pb["f0"]).ravel()[::97])
    return (np.concatenate([pb["w_true"] for pb in probs]), np.concatenate([pb["c_ref"] for pb in probs]),
            np.concatenate(parts))


# Tumour centroids at the planted coefficients (the truth of mm_error), found
# by the FP64 oracle's localisation and stored by tests/golden/make_bench_truth.py
# with a fingerprint of the inputs they belong to.
TRUTH_FILE = os.path.join(ROOT, "tests", "golden", "bench_truth.json")


def input_fingerprint(trace, c_ref, U):
    """Samples of the inputs a stored truth belongs to: every 7th row of the
    planted trace, the tumour centre and about 200 values of the eigenvector
    fields (inputs only: no arithmetic of the method).  Compared with a
    relative tolerance, so that last-bit differences of another machine's
    math library do not count as other inputs."""
    tr = np.asarray(trace, dtype=np.float64).reshape(len(trace), -1)
    u = np.asarray(U, dtype=np.float64).ravel()
    return {"trace": tr[::7].ravel().tolist(), "c_ref": np.asarray(c_ref, dtype=np.float64).ravel().tolist(),
            "U": u[:: max(1, u.size // 200)].tolist()}


def same_inputs(a, b, rtol=1e-5):
    return all(k in a and k in b and len(a[k]) == len(b[k]) and
               np.allclose(a[k], b[k], rtol=rtol, atol=rtol * max(1e-12, float(np.abs(b[k]).max(initial=0.0))))
               for k in ("trace", "c_ref", "U"))


def truth(name, trace, c_ref, U):
    """Stored oracle truth of workload `name` for these inputs, (T, 3) mm."""
    try:
        rec = json.load(open(TRUTH_FILE))[name]
    except (OSError, KeyError, ValueError) as e:
        raise SystemExit(f"no stored truth for {name} ({e}): run tests/golden/make_bench_truth.py")
    if not same_inputs(input_fingerprint(trace, c_ref, U), rec["fingerprint"]):
        raise SystemExit(f"stored truth for {name} belongs to other inputs: run tests/golden/make_bench_truth.py")
    return np.asarray(rec["c_true"], dtype=np.float64)


def view(angle):
    from paper_1102_1712_gb300 import synth as S
    d = WORKLOAD["det"]
    return S.cone_beam(d[0], d[1], d[2], d[3], float(angle))


def step_mm():
    v = WORKLOAD["vol"]
    return 0.5 * min(v[3], v[4], v[5])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------- algorithmic bytes
# size of the per-projection result record a queued solve copies back
SEQ_OUT_BYTES = 8 * 8 + 4 * 8 + 5 * 8 + 4 * 4


def kernel_bytes(N, M, K, has_mean):
    """Algorithmic HBM bytes per launch of each solver kernel (float32)."""
    model = 12 * K * N + (12 * N if has_mean else 0)
    return {
        "warp_pca": model + 4 * N + 4 * N,           # model read, f0 read once, f written
        "warp_batch": model + 4 * N + 20 * N,        # model + f0 once, five candidate volumes written
        "drr_solver": 4 * N + 4 * M + 4 * M,         # f read once, y read, p written
        "drr_batch": 20 * N + 4 * M + 20 * M,        # five volumes read once, y read, five p written
        "resid": 4 * M + 4 * M + 32 * M,             # p, y read; ray table written
        "adjoint_grad": model + 4 * N + 32 * M,      # model + f0 re-read; ray table read
    }


def first_gradient_bytes(kb, counts, N, K, has_mean):
    """Per-launch bytes with the gradient passes whose Jacobian pass the first
    evaluation's warp did (one per first-evaluation warp, labelled warp_pca:
    that warp reads the model and f0 once for both) counted without those
    reads: the average over the gradient launches."""
    out = dict(kb)
    nw, na = counts.get("warp_pca", 0), counts.get("adjoint_grad", 0)
    if na:
        model = 12 * K * N + (12 * N if has_mean else 0)
        out["adjoint_grad"] = (na * kb["adjoint_grad"] - min(nw, na) * (model + 4 * N)) / na
    return out


KERNEL_FILE = {"warp_pca": "k_warp_jac", "warp_batch": "k_warp_batch", "drr_solver": "k_drr_solver",
               "drr_batch": "k_drr_solver_batch", "resid": "k_resid", "adjoint_grad": "k_adjoint_grad"}


KERNEL_SOURCES = {"warp_batch": ("pcas_warp.cu", "pcas_internal.cuh")}


def strip_comments(src):
    """C++ source with its comments removed and each run of white space
    collapsed to one blank, so that a change to comments or layout alone
    leaves the hash of a kernel's sources as it was."""
    out, code, i, n = [], [], 0, len(src)

    def flush():
        out.append(" ".join("".join(code).split()))
        code.clear()

    while i < n:
        c = src[i]
        if c in "\"'":                  # a literal: kept verbatim
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            flush()
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
            code.append(" ")
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            code.append(" ")
        else:
            code.append(c)
            i += 1
    flush()
    return " ".join(t for t in out if t)


def kernel_source_hash(kernel):
    """Hash of the code (comments and layout aside) of the files a kernel is
    built from; a profile summary records it when its counters are taken."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, ("pcas_project.cu", "pcas_internal.cuh")):
        src = open(os.path.join(ROOT, "paper_1102_1712_gb300", "csrc", f), encoding="utf-8").read()
        h.update(strip_comments(src).encode())
    return h.hexdigest()[:16]


def ncu_field(kernel, field, cast=int):
    """One field of the committed ncu summary of this kernel on the sequence
    workload (``field: value`` lines), or None when the kernel sources changed
    since that capture."""
    path = os.path.join(ROOT, "profiles", f"{KERNEL_FILE[kernel]}_sequence_256x256x100_K3_512x384.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in text.splitlines()
                  if line.startswith(("kernel_source_sha256_16:", field + ":")))
    if fields.get("kernel_source_sha256_16", "").strip() != kernel_source_hash(kernel):
        return None
    try:
        return cast(fields[field].strip())
    except (KeyError, ValueError):
        return None


def ncu_traffic(kernel):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    return ncu_field(kernel, "traffic_bytes_per_launch")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


# ------------------------------------------------------------- our arm
def run_ours(args, ws_, rank, local):
    import torch

    from paper_1102_1712_gb300 import build as B
    from paper_1102_1712_gb300 import pcasolve as P
    from paper_1102_1712_gb300 import synth as S

    if rank == 0 or not B.up_to_date():
        B.build()
    if ws_ > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vol, f0, c_ref, U, trace, train, angles = make_inputs(args.irregular)
    angles = fixed_angles(args, angles)
    K, N = WORKLOAD["K"], f0.size
    d = WORKLOAD["det"]
    M = d[0] * d[1]
    step = step_mm()
    tf0 = torch.from_numpy(f0.ravel()).to(dev)
    tU = torch.from_numpy(U.ravel()).to(dev)
    W_, K_ = args.warmup, args.steps
    n_used = W_ + K_
    if n_used > WORKLOAD["n_proj"]:
        raise SystemExit(f"warmup + steps must be <= {WORKLOAD['n_proj']}")
    # measured projections: the planted volume f(w_true(t)) rendered by Siddon's
    # projector (or the solver's own) in the library + seeded noise
    ys = torch.empty((n_used, M), dtype=torch.float32, device=dev)
    c_true = truth("sequence-irregular" if args.irregular else "sequence-regular", trace, c_ref, U)
    for t in range(n_used):
        f = P.warp_volume(tf0, P.pca_dvf(None, tU, trace[t], vol), vol)
        if args.projector == "siddon":
            p = P.drr_siddon(f, vol, view(angles[t]))
        else:
            p = P.drr_forward(f, vol, view(angles[t]), step)
        sigma = WORKLOAD["noise"] * float(p.abs().max())
        ys[t] = p + torch.from_numpy(S.gaussian_noise(M, sigma, seed=1000 * WORKLOAD["seeds"]["noise"] + t)).to(dev)
    c_lp = P.lp_fit(train, 2)
    prm = P.default_params(step)
    wsp = P.Workspace(vol, view(0.0), K, device=dev)
    torch.cuda.synchronize()

    # launch shapes of this size bucket, measured before anything is timed
    tune_s, tuning = 0.0, None
    if args.tuning:
        P.tuning_set(vol, view(0.0), K, json.loads(args.tuning))
    elif not args.no_autotune:
        t0 = time.perf_counter()
        tuning = P.autotune(tf0, None, tU, ys[0], vol, view(angles[0]), prm, w_init=trace[0], ws=wsp)
        tune_s = time.perf_counter() - t0
    else:
        P.tuning_clear()
    solver = P.Solver(tf0, None, tU, vol, view(0.0), prm, device=dev)
    view_cache = None
    if args.workload == "fluoro" and not args.no_view_cache:
        # Sec. IV: the gantry is held still, so the constant part of P^T (every
        # voxel's footprint and ray weights) is computed once and kept
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nbytes = solver.fix_view(float(angles[0]))
        torch.cuda.synchronize()
        view_cache = {"bytes": nbytes, "build_s": round(time.perf_counter() - t0, 3)}

    def solve_range(t0, t1, hist, y_of, stats_out):
        """Host-driven sequence driver (every kernel launched and timed from the
        host): Eq. (3) warm start, solve, localise, per projection."""
        for t in range(t0, t1):
            if t == 0:
                w0 = np.zeros(K)
            elif t == 1:
                w0 = hist[-1]
            else:
                w0 = P.lp_predict(np.stack([hist[-1], hist[-2]]), c_lp)
            w, st = P.solve_projection(tf0, None, tU, y_of(t), vol, view(angles[t]), w0, prm, ws=wsp)
            c, _ = P.localize_tumor(None, tU, w, vol, c_ref)
            hist.append(w)
            stats_out.append((t, st, c))

    # warm-up projections: the start of a run of the device-driven solver (the
    # Eq. 3 warm start and the localisation inside its graph), which the timed
    # projections continue; also builds the host-side history
    stream = torch.cuda.current_stream()
    solver.seq_begin(c_lp, c_ref)
    warm = solver.solve_sequence([ys[t] for t in range(W_)], angles[:W_], w_first=np.zeros(K))
    hist = [w for w, _, _, _ in warm]
    solve_range(0, 2, [], lambda t: ys[t], [])
    torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM, device-driven solves queued back to back
    P.profile(False)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if ws_ > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        res = solver.solve_sequence([ys[t] for t in range(W_, n_used)], angles[W_:n_used])
        ev1.record(stream)
        torch.cuda.synchronize()
        if ws_ > 1:
            torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    timed = [(W_ + i, st, c) for i, (w, st, c, _) in enumerate(res)]
    launches_timed = sum(n for n, _ in P.profile_read().values())
    clocks = clk.summary()
    if view_cache is not None:
        # the same run without the cache: bitwise the same solutions, every P^T
        # weight recomputed in each gradient
        solver.fix_view(None)
        solver.seq_begin(c_lp, c_ref, w_hist=[hist[W_ - 1], hist[W_ - 2]])
        torch.cuda.synchronize()
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        res_u = solver.solve_sequence([ys[t] for t in range(W_, n_used)], angles[W_:n_used])
        u1.record(stream)
        torch.cuda.synchronize()
        view_cache["uncached_value"] = round(K_ / (u0.elapsed_time(u1) / 1e3), 3)
        view_cache["same_solutions"] = all(np.array_equal(a[0], b[0]) for a, b in zip(res, res_u))
        solver.fix_view(float(angles[0]))

    # ---- the same projections host-driven, every kernel bracketed by CUDA events
    P.profile(True)
    timed_host = []
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    h0.record(stream)
    solve_range(W_, n_used, list(hist[:W_]), lambda t: ys[t], timed_host)
    h1.record(stream)
    torch.cuda.synchronize()
    ms_host = h0.elapsed_time(h1)
    prof = P.profile_read()
    P.profile(False)

    # ---- end to end: per step, y copied from pinned host memory inside the
    # queued solve and its result record read back to pinned host memory
    y_host = ys.cpu().pin_memory()
    solver.seq_begin(c_lp, c_ref, w_hist=[hist[W_ - 1], hist[W_ - 2]])
    if ws_ > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res_e2e = solver.solve_sequence([y_host[t] for t in range(W_, n_used)], angles[W_:n_used])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    if ws_ > 1:
        torch.distributed.barrier()

    # ---- aggregate over ranks (max time)
    t_s, te_s = max_over_ranks([ms / 1e3, ms_e2e / 1e3], ws_, dev)
    if rank != 0:
        return None

    errs = np.array([np.linalg.norm(c - c_true[t]) for t, _, c in timed])
    iters = np.array([st["iters"] for _, st, _ in timed])
    evals = np.array([st["evals"] for _, st, _ in timed])
    pk, pk_kind = peaks()
    kb = first_gradient_bytes(kernel_bytes(N, M, K, has_mean=False), {k: prof[k][0] for k in prof}, N, K, False)
    kernels = {}
    for name in ("warp_pca", "warp_batch", "drr_solver", "drr_batch", "resid", "adjoint_grad"):
        n, tot = prof[name]
        if n:
            avg = tot / n
            gbs = kb[name] / (avg * 1e-3) / 1e9
            kernels[name] = {"launches": n, "total_ms": round(tot, 3), "avg_ms": round(avg, 4),
                             "share": round(tot / ms_host, 4), "alg_bytes": int(kb[name]),
                             "achieved_gbs": round(gbs, 1), "frac_hbm": round(gbs / pk["hbm_gbs"], 4)}
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
    launches = launches_timed
    # the whole path in the one-at-a-time accounting of the method: per
    # projection iters gradient evaluations of B_g bytes and (evals - 1) trial
    # evaluations of B_t bytes, over the device-driven run's time; the motion
    # model is read twice per gradient evaluation and once per trial (12 bytes
    # per voxel and field: the K eigenvectors, and the mean only where there is one)
    has_mean = False
    nf = K + (1 if has_mean else 0)
    B_g = (24 * nf + 12) * N + 16 * M
    B_t = (12 * nf + 12) * N + 4 * M
    B_path = float(np.sum(iters * B_g + (evals - 1) * B_t))
    path_run_gbs = B_path / (ms / 1e3) / 1e9
    total_alg = sum(kernels[k]["alg_bytes"] * kernels[k]["launches"] for k in kernels)
    line = {
        "metric": METRIC,
        "value": round(replica_throughput(ws_, K_, t_s), 3),
        "unit": "projections/s",
        "n_gpus": ws_,
        "steps": K_,
        "warmup": W_,
        "ms_per_step": round(1e3 * t_s / K_, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded ellipsoid phantom, smoothed random eigen-DVFs, sinusoidal trace; "
                f"projections rendered by this library's {args.projector} projector + 1% noise)",
        "config": {"workload": workload_name(args),
                   "volume": "256x256x100 @ 2x2x2.5 mm", "K": K, "detector": "512x384 @ 0.776 mm",
                   "step_mm": step,
                   "projections": (f"{W_}+{K_} of 600 at {args.angle_deg:g} deg" if args.workload == "fluoro"
                                   else f"{W_}+{K_} of 600 over 360 deg"),
                   "measured_images": args.projector,
                   "solver": "mu0=0.2 alpha=0.1 beta=0.5 mu_min=0.01 max_iter=10",
                   "l2": "inputs larger than L2 (motion model 236 MB streamed per evaluation)",
                   "parallelism": "replicas" if ws_ > 1 else "single"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["achieved_gbs"],
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": kernels[dom]["frac_hbm"],
                     "traffic": ncu_traffic(dom), "peak_source": pk_kind,
                     "l1_pipe_frac": ncu_field(dom, "l1tex_throughput_frac", float),
                     "smem_wavefront_frac": ncu_field(dom, "smem_wavefront_frac", float),
                     "issue_active_frac": ncu_field(dom, "issue_active_frac", float),
                     "path_alg_gbs": round(total_alg / (ms_host / 1e3) / 1e9, 1),
                     "path_frac": round(total_alg / (ms_host / 1e3) / 1e9 / pk["hbm_gbs"], 4),
                     "path_bytes": "the bytes the kernels move (sum over launches of each kernel's algorithmic "
                                   "bytes), over the host-driven pass's time",
                     "run_path_gbs": round(path_run_gbs, 1),
                     "run_path_frac": round(path_run_gbs / pk["hbm_gbs"], 4),
                     "run_path_bytes": "the method's one-at-a-time accounting: per projection iters * "
                                       "((24K+12)N + 16M) + (evals-1) * ((12K+12)N + 4M) (no mean field), over "
                                       "the device-driven run's time; the batched line search moves fewer bytes "
                                       "than this counts",
                     "note": "kernel durations from CUDA events in the host-driven pass over the same "
                             "projections (graph launches cannot be bracketed per kernel)"},
        "host_driven": {"value": round(K_ / (ms_host / 1e3), 3), "ms_per_step": round(ms_host / K_, 4)},
        **({"view_cache": view_cache} if view_cache is not None else {}),
        "launch_shapes": {"autotuned": tuning is not None, "given": bool(args.tuning), "tune_s": round(tune_s, 2),
                          "entry": tuning or P.tuning_get(vol, view(0.0), K)},
        "kernels": kernels,
        "gpu_launches": launches,
        "clocks": clocks,
        "mm_error": {"mean": round(float(errs.mean()), 4), "p95": round(float(np.percentile(errs, 95)), 4),
                     "max": round(float(errs.max()), 4)},
        "solver": {"iters_mean": round(float(iters.mean()), 3), "evals_mean": round(float(evals.mean()), 3)},
        "e2e": {"value": round(replica_throughput(ws_, K_, te_s), 3), "unit": "projections/s",
                "h2d_bytes_per_step": 4 * M,
                # the projection's result record (solution, centroid, statistics)
                "d2h_bytes_per_step": SEQ_OUT_BYTES},
    }
    if ws_ == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], o = cpu_baseline(vol, f0, c_ref, U, trace, train, angles, ys, W_)
        # the same projection from the same start on the GPU: parity at full size
        w_g, st_g = P.solve_projection(tf0, None, tU, ys[W_], vol, view(angles[W_]), o["w0"], prm, ws=wsp)
        c_g, _ = P.localize_tumor(None, tU, w_g, vol, c_ref)
        line["oracle_parity"] = {"projection": W_, "w_max_abs_diff": float(np.abs(w_g - o["w"]).max()),
                                 "centroid_diff_mm": float(np.linalg.norm(c_g - o["c"])),
                                 "J_rel_diff": float(abs(st_g["J"] - o["J"]) / o["J"]),
                                 "iters_gpu_oracle": [st_g["iters"], o["iters"]],
                                 "evals_gpu_oracle": [st_g["evals"], o["evals"]]}
    return line


# ------------------------------------------------------- oracle timings
def oracle_solve_one(O, vol, f0, U, y, angle, w0, step):
    from paper_1102_1712_gb300 import synth as S  # noqa: F401  (inputs only)
    prm = dict(mu0=0.2, alpha=0.1, beta=0.5, mu_min=0.01, max_iter=10, max_trials=30, step=step)
    return O.solve_projection(f0, None, U, y, vol, view(angle), w0, prm)


def cpu_baseline(vol, f0, c_ref, U, trace, train, angles, ys, t):
    """The oracle (FP64 C, OpenMP over rays) solving one projection of the
    workload, warm-started from the prediction of the planted coefficients."""
    import oracle as O
    c_lp = O.lp_fit(train, 2)
    w0 = O.lp_predict(np.stack([trace[t - 1], trace[t - 2]]), c_lp)
    y = ys[t].cpu().numpy()
    t0 = time.perf_counter()
    w, st, _ = oracle_solve_one(O, vol, f0, U, y, angles[t], w0, step_mm())
    c, _ = O.localize_tumor(None, U, w, vol, c_ref)
    dt = time.perf_counter() - t0
    line = {"value": round(1.0 / dt, 5), "unit": "projections/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 projection (#{t}) of the same workload, full solve ({st['iters']} iterations, "
                      f"{st['evals']} evaluations) + localisation, {dt:.1f} s; OpenMP over the rays of the "
                      "forward projector and the voxels of the DVF and warp, the P^T scatter and the "
                      "gradient reduction serial (their sums in written order)"}
    return line, {"w0": w0, "w": np.asarray(w), "c": np.asarray(c), "J": st["J"], "iters": st["iters"],
                  "evals": st["evals"]}


def run_reference(args, ws_, rank):
    """Oracle arm: solves projections of the workload on the host cores, each
    warm-started from the prediction of the planted coefficients, until
    ``steps`` projections or 150 s of solving are done (bounded sample)."""
    if rank != 0:
        return None
    import oracle as O
    from paper_1102_1712_gb300 import synth as S
    O.build()
    vol, f0, c_ref, U, trace, train, angles = make_inputs(args.irregular)
    angles = fixed_angles(args, angles)
    step = step_mm()
    c_lp = O.lp_fit(train, 2)
    done, t_total, t_limit = 0, 0.0, 150.0
    for i in range(args.warmup + args.steps):
        t = 2 + i
        cb = view(angles[t])
        f_true = O.warp_volume(f0, O.pca_dvf(None, U, trace[t], vol), vol)
        if args.projector == "siddon":
            p = O.siddon_forward(f_true, vol, cb)
        else:
            p = O.drr_forward(f_true, vol, cb, step)
        y = (p + S.gaussian_noise(p.size, WORKLOAD["noise"] * np.abs(p).max(),
                                  seed=1000 * WORKLOAD["seeds"]["noise"] + t, dtype=np.float64)).astype(np.float32)
        w0 = O.lp_predict(np.stack([trace[t - 1], trace[t - 2]]), c_lp)
        t0 = time.perf_counter()
        w, st, _ = oracle_solve_one(O, vol, f0, U, y, angles[t], w0, step)
        O.localize_tumor(None, U, w, vol, c_ref)
        dt = time.perf_counter() - t0
        if i >= args.warmup or args.warmup + args.steps == 1:
            done += 1
            t_total += dt
        if t_total > t_limit or (i < args.warmup and dt > t_limit / 4):
            break
    done = max(done, 1)
    t_total = max(t_total, 1e-9)
    value = done / t_total
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "projections/s",
            "n_gpus": 1, "steps": done, "warmup": args.warmup, "ms_per_step": round(1e3 * t_total / done, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic, same workload as our arm", "config": {"workload": workload_name(args)},
            "cpu_baseline": {"value": round(value, 5), "unit": "projections/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{done} projection{'s' if done != 1 else ''} of the workload, full solves, "
                                       "at most about 150 s of solving; OpenMP over the rays of the forward projector "
                                       "and the voxels of the DVF and warp, the P^T scatter and the gradient "
                                       "reduction serial"},
            "e2e": {"value": round(value, 5), "unit": "projections/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------- precision workload
def run_precision(args, local):
    import torch

    from paper_1102_1712_gb300 import build as B
    from paper_1102_1712_gb300 import pcasolve as P
    from paper_1102_1712_gb300 import synth as S

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = PRECISION
    vol, f0, c_ref, U, trace, train, angles = precision_inputs()
    d = W["det"]
    views = [S.cone_beam(d[0], d[1], d[2], d[3], float(a)) for a in angles]
    step = 0.5 * min(W["vol"][3:])
    K, M = W["K"], d[0] * d[1]
    W_, K_ = args.warmup, args.steps
    n_used = W_ + K_
    tf0 = torch.from_numpy(f0.ravel()).to(dev)
    tU = torch.from_numpy(U.ravel()).to(dev)
    ys = torch.empty((n_used, M), dtype=torch.float32, device=dev)
    c_true = truth("precision", trace, c_ref, U)
    for t in range(n_used):
        f = P.warp_volume(tf0, P.pca_dvf(None, tU, trace[t], vol), vol)
        p = P.drr_siddon(f, vol, views[t]) if args.projector == "siddon" else P.drr_forward(f, vol, views[t], step)
        sigma = W["noise"] * float(p.abs().max())
        ys[t] = p + torch.from_numpy(S.gaussian_noise(M, sigma, seed=1000 * W["seeds"]["noise"] + t)).to(dev)
    c_lp = P.lp_fit(train, 2)
    prm = P.default_params(step)
    wsp = P.Workspace(vol, views[0], K, device=dev)
    kb = kernel_bytes(f0.size, M, K, False)
    out = {}
    pk, pk_kind = peaks()
    for name, dt in [("float32", torch.float32), ("bfloat16", torch.bfloat16), ("float16", torch.float16)]:
        sf0, sU = tf0.to(dt), tU.to(dt)
        if not args.no_autotune:
            P.autotune(sf0, None, sU, ys[0], vol, views[0], prm, w_init=trace[0], ws=wsp)
        solver = P.Solver(sf0, None, sU, vol, views[0], prm, device=dev)
        stream = torch.cuda.current_stream()
        # warm-up projections start the device-driven run the timed ones continue
        solver.seq_begin(c_lp, c_ref)
        warm = solver.solve_sequence([ys[t] for t in range(W_)], angles[:W_], w_first=np.zeros(K))
        hist = [w for w, _, _, _ in warm]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            res = solver.solve_sequence([ys[t] for t in range(W_, n_used)], angles[W_:n_used])
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        solver.close()
        timed = [(W_ + i, st, c) for i, (w, st, c, _) in enumerate(res)]

        # the same projections host-driven, every kernel bracketed by CUDA events
        def solve(t, h, rec):
            w0 = np.zeros(K) if t == 0 else h[-1] if t == 1 else P.lp_predict(np.stack([h[-1], h[-2]]), c_lp)
            w, st = P.solve_projection(sf0, None, sU, ys[t], vol, views[t], w0, prm, ws=wsp)
            c, _ = P.localize_tumor(None, sU, w, vol, c_ref)
            h.append(w)
            rec.append((t, st, c))

        P.profile(True)
        hh, timed_host = list(hist), []
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        h0.record(stream)
        for t in range(W_, n_used):
            solve(t, hh, timed_host)
        h1.record(stream)
        torch.cuda.synchronize()
        ms_host = h0.elapsed_time(h1)
        prof = P.profile_read()
        P.profile(False)
        errs = np.array([np.linalg.norm(c - c_true[t]) for t, _, c in timed])
        # model and CT bytes scale with the storage size (warp and Jacobian passes)
        scale = {"float32": 1.0, "bfloat16": 0.5, "float16": 0.5}[name]
        kbs = first_gradient_bytes(kb, {k: prof[k][0] for k in prof}, f0.size, K, False)
        kern = {}
        for kname in ("warp_pca", "warp_batch", "drr_solver", "drr_batch", "resid", "adjoint_grad"):
            n, tot = prof[kname]
            if n:
                by = kbs[kname]
                if kname in ("warp_pca", "warp_batch", "adjoint_grad"):
                    # the share of launches that read the model and f0
                    nw, na = prof["warp_pca"][0], prof["adjoint_grad"][0]
                    reads = (na - min(nw, na)) / na if kname == "adjoint_grad" and na else 1.0
                    by = int(by - (1.0 - scale) * (12 * K + 4) * f0.size * reads)
                kern[kname] = {"launches": n, "avg_ms": round(tot / n, 4), "share": round(tot / ms_host, 4),
                               "achieved_gbs": round(by / (tot / n * 1e-3) / 1e9, 1)}
        out[name] = {"value": round(K_ / (ms / 1e3), 3), "ms_per_step": round(ms / K_, 4),
                     "host_driven": round(K_ / (ms_host / 1e3), 3),
                     "mm_error": {"mean": round(float(errs.mean()), 4), "p95": round(float(np.percentile(errs, 95)), 4),
                                  "max": round(float(errs.max()), 4)},
                     "kernels": kern, "clocks": clk.summary(),
                     "centroids": [c.tolist() for _, _, c in timed]}
        del sf0, sU
    # 16-bit storage against float32 at the same projections
    cf = np.array(out["float32"].pop("centroids"))
    for name in ("bfloat16", "float16"):
        cl = np.array(out[name].pop("centroids"))
        out[name]["centroid_vs_float32_mm_max"] = round(float(np.abs(cl - cf).max()), 5)
    bf = out["bfloat16"]
    dom = max(bf["kernels"], key=lambda k: bf["kernels"][k]["share"])
    return {"metric": METRIC, "value": bf["value"], "unit": "projections/s", "n_gpus": 1, "steps": K_,
            "warmup": W_, "ms_per_step": bf["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 storage, f32 arithmetic",
            "data": "synthetic (seeded phantom, coarse-grid smoothed eigen-DVFs, irregular trace; "
                    f"projections rendered by this library's {args.projector} projector + 1% noise)",
            "config": {"workload": W["name"], "volume": "512x512x160 @ 1x1x2 mm", "K": K,
                       "detector": "1024x768 @ 0.388 mm", "step_mm": step,
                       "projections": f"{W_}+{K_} of 300 over 360 deg, irregular"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": bf["kernels"][dom]["achieved_gbs"],
                         "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": round(bf["kernels"][dom]["achieved_gbs"] / pk["hbm_gbs"], 4),
                         "traffic": None, "peak_source": pk_kind},
            "storage": out, "clocks": bf["clocks"]}


# ----------------------------------------------------------- batch workload
def run_batch(args, local):
    import torch

    from paper_1102_1712_gb300 import build as B
    from paper_1102_1712_gb300 import pcasolve as P
    from paper_1102_1712_gb300 import synth as S

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = BATCH
    models = {}
    probs = batch_inputs()
    c_true_all = truth("batch", *batch_fingerprint_parts(probs))
    for i, pb in enumerate(probs):
        pb["c_true"] = c_true_all[i]
        key = pb["model"]
        if key not in models:
            models[key] = torch.from_numpy(pb["U"].ravel()).to(dev)
        pb["U"] = models[key]
        pb["f0"] = torch.from_numpy(pb["f0"].ravel()).to(dev)
    for i, pb in enumerate(probs):
        M = pb["cb"]["nu"] * pb["cb"]["nv"]
        f = P.warp_volume(pb["f0"], P.pca_dvf(None, pb["U"], pb["w_true"], pb["vol"]), pb["vol"])
        p = (P.drr_siddon(f, pb["vol"], pb["cb"]) if args.projector == "siddon"
             else P.drr_forward(f, pb["vol"], pb["cb"], pb["step"]))
        sigma = W["noise"] * float(p.abs().max())
        pb["y"] = p + torch.from_numpy(S.gaussian_noise(M, sigma, seed=300 + i)).to(dev)
        pb["prm"] = P.default_params(pb["step"], max_iter=20)     # cold starts: 20 iterations, as the tiny case
    # one autotune per size bucket (volume, detector, K), on its first problem
    t0 = time.perf_counter()
    tuned = {}
    for pb in probs:
        key = (pb["vol"]["nx"], pb["cb"]["nu"], pb["K"])
        if key in tuned or args.no_autotune:
            continue
        ws_t = P.Workspace(pb["vol"], pb["cb"], pb["K"], device=dev)
        tuned[key] = P.autotune(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], pb["prm"], ws=ws_t)
        del ws_t
    if args.no_autotune:
        P.tuning_clear()
    tune_s = time.perf_counter() - t0
    solvers = [P.Solver(pb["f0"], None, pb["U"], pb["vol"], pb["cb"], pb["prm"], device=dev) for pb in probs]
    batch = P.Batch(solvers, ys=[pb["y"] for pb in probs])
    angles = [pb["cb"]["angle"] for pb in probs]
    w_init = [np.zeros(pb["K"]) for pb in probs]
    wsps = [P.Workspace(pb["vol"], pb["cb"], pb["K"], device=dev) for pb in probs]
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = None
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    def one_after_another_host():
        return [P.solve_projection(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], np.zeros(pb["K"]),
                                   pb["prm"], ws=wsps[i]) for i, pb in enumerate(probs)]

    def one_after_another_graph():
        return [sv.solve(pb["y"], np.zeros(pb["K"])) for sv, pb in zip(solvers, probs)]

    reps = max(1, args.steps)
    for _ in range(max(args.warmup, 1)):
        batch.solve(angles, w_init)
    one_after_another_host()
    P.profile(False)                             # reset the launch counters
    with ClockSampler(local) as clk:
        ms_b, (ws, sts) = timed(lambda: batch.solve(angles, w_init), reps)
    launches = sum(n for n, _ in P.profile_read().values())
    ms_s, seq = timed(one_after_another_host, reps)
    ms_g, _ = timed(one_after_another_graph, reps)
    # per-kernel roofline: each problem's host-driven solve with every kernel
    # bracketed by CUDA events, bytes from that problem's own sizes
    pk, pk_kind = peaks()
    agg = {}
    for i, pb in enumerate(probs):
        P.profile(True)
        P.solve_projection(pb["f0"], None, pb["U"], pb["y"], pb["vol"], pb["cb"], np.zeros(pb["K"]), pb["prm"],
                           ws=wsps[i])
        prof = P.profile_read()
        P.profile(False)
        v = pb["vol"]
        nv = v["nx"] * v["ny"] * v["nz"]
        kb = first_gradient_bytes(kernel_bytes(nv, pb["cb"]["nu"] * pb["cb"]["nv"], pb["K"], has_mean=False),
                                  {k: prof[k][0] for k in prof}, nv, pb["K"], False)
        for name in kb:
            cnt, tot = prof[name]
            a = agg.setdefault(name, [0, 0.0, 0.0])
            a[0] += cnt
            a[1] += tot
            a[2] += cnt * kb[name]
    kern = {name: {"launches": c, "total_ms": round(t, 3), "alg_bytes": int(by),
                   "achieved_gbs": round(by / (t * 1e-3) / 1e9, 1), "frac_hbm": round(by / (t * 1e-3) / 1e9 / pk["hbm_gbs"], 4)}
            for name, (c, t, by) in agg.items() if c}
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["achieved_gbs"], "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": kern[dom]["frac_hbm"], "traffic": None, "peak_source": pk_kind,
                "note": "host-driven solves of the 64 problems, every kernel bracketed by CUDA events"}
    n = W["n"]
    errs = []
    for i, pb in enumerate(probs):
        c, _ = P.localize_tumor(None, pb["U"], ws[i], pb["vol"], pb["c_ref"])
        errs.append(np.linalg.norm(c - pb["c_true"]))
        assert np.array_equal(ws[i], seq[i][0]), "batched and sequential solves disagree"
    errs = np.array(errs)
    value = n * reps / (ms_b / 1e3)
    return {"metric": METRIC, "value": round(value, 3), "unit": "projections/s", "n_gpus": 1, "steps": reps,
            "warmup": max(args.warmup, 1), "ms_per_step": round(ms_b / reps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (64 seeded phantoms, 6 seeded eigenvector models, random angles, w ~ N(0,1); "
                    f"projections rendered by this library's {args.projector} projector + 1% noise)",
            "config": {"workload": W["name"], "solves_per_step": n,
                       "volumes": "128^2x64 / 192^2x96 / 256^2x128", "K": "3 / 5",
                       "detectors": "256x192 / 512x384 / 768x576 / 1024x768", "start": "w = 0",
                       "solver": "mu0=0.2 alpha=0.1 beta=0.5 mu_min=0.01 max_iter=20"},
            "one_after_another": {"host_driven": round(n * reps / (ms_s / 1e3), 3),
                                  "graph_per_solve": round(n * reps / (ms_g / 1e3), 3), "unit": "projections/s"},
            "speedup_vs_host_driven": round(ms_s / ms_b, 3),
            "mm_error": {"mean": round(float(errs.mean()), 4), "p95": round(float(np.percentile(errs, 95)), 4),
                         "max": round(float(errs.max()), 4)},
            "solver": {"iters_mean": round(float(np.mean([s["iters"] for s in sts])), 3),
                       "evals_mean": round(float(np.mean([s["evals"] for s in sts])), 3)},
            "launch_shapes": {"autotuned_buckets": len(tuned), "tune_s": round(tune_s, 2)},
            "roofline": roofline, "kernels": kern,
            "gpu_launches": launches, "clocks": clk.summary()}


# ------------------------------------------------------- oracle timings per config
def run_oracle_timing(args):
    """The FP64 oracle on the host cores: per evaluation (cost_grad, median of
    three) on the tiny, sequence and precision volumes, and per projection
    (full solve + localisation) on the tiny case and on --steps projections of
    the sequence (every 30th from #5, warm-started from the prediction of the
    planted coefficients).  Measured images rendered by the oracle's Siddon
    projector.  Bounded: a few minutes on 16 cores."""
    import oracle as O
    from paper_1102_1712_gb300 import synth as S
    O.build()

    def med3(fn):
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts))

    out = {"impl": "oracle-timing", "kind": "oracle", "cores": os.cpu_count(), "unit": "s"}
    # tiny: 64x64x32 at 4 mm, K = 3, 128x96 at 3.1 mm, 20 iterations from w = 0
    vol = S.volume(64, 64, 32, 4.0, 4.0, 4.0)
    f0, c_ref = S.phantom(vol, 15.0, seed=1)
    U = S.eigen_dvfs(vol, 3, seed=2)
    cb = S.cone_beam(128, 96, 3.1, 3.1, 0.0)
    w_true = np.array([1.2, -0.4, 0.3])
    y = O.siddon_forward(O.warp_volume(f0, O.pca_dvf(None, U, w_true, vol), vol), vol, cb)
    y = (y + S.gaussian_noise(y.shape, 0.01 * np.abs(y).max(), seed=3, dtype=np.float64)).astype(np.float32)
    prm = dict(mu0=0.2, alpha=0.1, beta=0.5, mu_min=0.01, max_iter=20, max_trials=30, step=2.0)
    t_eval = med3(lambda: O.cost_grad(f0, None, U, 0.5 * w_true, y, vol, cb, 2.0))
    t0 = time.perf_counter()
    _, st, _ = O.solve_projection(f0, None, U, y, vol, cb, np.zeros(3), prm)
    O.localize_tumor(None, U, _, vol, c_ref)
    out["tiny"] = {"eval_s": round(t_eval, 4), "projection_s": round(time.perf_counter() - t0, 3),
                   "iters": st["iters"], "evals": st["evals"]}
    # sequence: 256x256x100, K = 3, 512x384
    vol, f0, c_ref, U, trace, train, angles = make_inputs(False)
    step = step_mm()
    c_lp = O.lp_fit(train, 2)
    ts = [5 + 30 * i for i in range(max(1, args.steps))]
    y0 = None
    proj = []
    for t in ts:
        f = O.warp_volume(f0, O.pca_dvf(None, U, trace[t], vol), vol)
        y = O.siddon_forward(f, vol, view(angles[t]))
        y = (y + S.gaussian_noise(y.shape, WORKLOAD["noise"] * np.abs(y).max(),
                                  seed=1000 * WORKLOAD["seeds"]["noise"] + t, dtype=np.float64)).astype(np.float32)
        if y0 is None:
            y0 = (y, t)
        w0 = O.lp_predict(np.stack([trace[t - 1], trace[t - 2]]), c_lp)
        t0 = time.perf_counter()
        w, st, _ = oracle_solve_one(O, vol, f0, U, y, angles[t], w0, step)
        O.localize_tumor(None, U, w, vol, c_ref)
        proj.append({"projection": t, "s": round(time.perf_counter() - t0, 3), "iters": st["iters"],
                     "evals": st["evals"]})
    y, t = y0
    t_eval = med3(lambda: O.cost_grad(f0, None, U, trace[t], y, vol, view(angles[t]), step))
    out["sequence"] = {"eval_s": round(t_eval, 3), "projections": proj,
                       "projections_per_s": round(len(proj) / sum(p["s"] for p in proj), 5)}
    # precision volume: 512x512x160 at 1x1x2 mm, K = 5, 1024x768 (one evaluation)
    W = PRECISION
    vol = S.volume(*W["vol"])
    f0, c_ref = S.phantom(vol, W["tumor_mm"], seed=W["seeds"]["phantom"])
    U = S.eigen_dvfs(vol, W["K"], seed=W["seeds"]["dvf"], coarse=(2, 4, 4))
    d = W["det"]
    cb = S.cone_beam(d[0], d[1], d[2], d[3], 0.4)
    w5 = np.array([1.0, 0.3, 0.15, 0.1, -0.05])
    y = O.siddon_forward(O.warp_volume(f0, O.pca_dvf(None, U, w5, vol), vol), vol, cb).astype(np.float32)
    t0 = time.perf_counter()
    O.cost_grad(f0, None, U, 0.8 * w5, y, vol, cb, 0.5 * min(W["vol"][3:]))
    out["precision"] = {"eval_s": round(time.perf_counter() - t0, 3)}
    return out


def extra_workloads(args, local):
    """The batch and precision workloads in short form beside the sequence
    line: 64 uneven solves in one launch (one warm-up launch, one timed), and
    3 + 10 projections of the precision workload per storage type.  Each
    sub-object keeps its throughput, roofline of the dominant kernel, mm error
    and clocks; about a minute of set-up and timing together."""
    import copy
    out = {}
    a = copy.copy(args)
    a.steps, a.warmup = 1, 1
    b = run_batch(a, local)
    out["batch"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "one_after_another", "speedup_vs_host_driven",
                                      "mm_error", "solver", "gpu_launches", "clocks")}
    out["batch"]["workload"] = b["config"]["workload"]
    if "roofline" in b:
        out["batch"]["roofline"] = b["roofline"]
    a = copy.copy(args)
    a.steps, a.warmup = 10, 3
    p = run_precision(a, local)
    out["precision"] = {"workload": p["config"]["workload"], "unit": "projections/s", "roofline": p["roofline"],
                        "clocks": p["clocks"],
                        "storage": {k: {kk: v[kk] for kk in ("value", "ms_per_step", "mm_error", "kernels") if kk in v}
                                    | ({"centroid_vs_float32_mm_max": v["centroid_vs_float32_mm_max"]}
                                       if "centroid_vs_float32_mm_max" in v else {})
                                    for k, v in p["storage"].items()}}
    return out


def main():
    args = parse()
    ws_, rank, local = dist_env()
    if ws_ > 1 and args.impl == "ours":
        import torch
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        line = run_reference(args, ws_, rank)
    elif args.workload == "precision":
        line = run_precision(args, local) if rank == 0 else None
    elif args.workload == "batch":
        line = run_batch(args, local) if rank == 0 else None
    elif args.workload == "oracle":
        line = run_oracle_timing(args) if rank == 0 else None
    else:
        line = run_ours(args, ws_, rank, local)
        if line is not None and ws_ == 1 and args.workload == "sequence" and not args.no_extra:
            line.update(extra_workloads(args, local))
    if line is not None:
        print(json.dumps(line), flush=True)
    if ws_ > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
