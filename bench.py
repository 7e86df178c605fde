"""Benchmark of the joint pose-appearance training step (one iteration of
Algorithm 1 over a batch of views: projection, tile sort, compositing,
fused L1 + backward with pose gradient, Huber track term, Adam on
Gaussians, track points and SE(3) pose deltas).

Default workload (`large`): 1000 cameras of uneven resolution (960..1920 x
540..1080) on a sphere looking at the scene, 5M Gaussians with SH degree 3,
400k tracks with 2..40 observations each over the views that see them; each
step trains on 16 random views, batched (one launch per stage for all 16,
the batch laid out on the device) and captured in one CUDA graph.  Other
workloads: train (8 of 200 views 1600x1066, 3M Gaussians), batched (32
uneven views, 1M), mid (8 views 1237x822, 200k).  Prints one JSON line
(metric: Mpix*views/s of the joint fwd+bwd step).

--impl reference times the FP64 CPU oracle (the paper publishes no code to
compare against) on a bounded pixel sample of the same workload, over all
host cores.
--gpus N under torchrun runs N independent replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402  (seeded random draws only)

METRIC = "joint fwd+bwd steps/s (Mpix·views/s) incl. pose+track grads; % HBM roofline"
UNIT = "Mpix*views/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "train", "batched", "mid", "sfm-ba", "mcmc"],
                    help="large (default): 16 random views of 1000 uneven ones (960-1920 x 540-1080), 5M "
                         "Gaussians; sfm-ba: Levenberg-Marquardt iterations of the bundle adjustment of Eq. 4; "
                         "mcmc: the MCMC densification step on 3M Gaussians")
    ap.add_argument("--mode", default="batched", choices=["batched", "plain"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain one-view-per-launch timing")
    ap.add_argument("--lambda-ssim", type=float, default=0.0,
                    help="SSIM weight of Eq. 5 (the paper: 0.2); 0 = the L1 photometric term alone")
    ap.add_argument("--variant", default="full", choices=["full", "frozen-poses", "photometric-only", "merged-tracks"],
                    help="the paper's ablation variants of the joint step (full: the method)")
    ap.add_argument("--deterministic", action="store_true",
                    help="the compositing backward with run-to-run bit-identical gradients")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run this many eager steps and exit (for ncu launch lists)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_desc(name, w):
    W = w["workload"]
    return dict(workload="%s: %d views %s, %d Gaussians SH%d, %d tracks (%d-%d obs), batch %d" % (
        name, W.n_views, "%dx%d" % (W.width[0], W.height[0]) if W.width[0] == W.width[1] else
        "%d-%dx%d-%d" % (W.width[0], W.width[1], W.height[0], W.height[1]), W.n_gaussians, W.sh_degree,
        W.n_tracks, W.obs_range[0], W.obs_range[1], W.batch))


# ---------------------------------------------------------------------------
# CPU oracle leg: the FP64 oracle as it stands, timed on a bounded sample of
# the workload, on one spawned process per host core.  Each process renders
# its own share of the sampled pixels (forward and backward over all
# Gaussians, per pixel by brute force); the scene's arrays are written once
# as .npy files that every process maps read-only.

SCENE_KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def np_visible(X, wh, K, Rt, near=0.01):
    """bool [n, V]: point X_k in view v's image with depth > near (pinhole
    projection of the track points, used to draw the track observations)."""
    R = np.asarray(Rt)[:, :9].reshape(-1, 3, 3)
    t = np.asarray(Rt)[:, 9:]
    Xc = np.einsum("vij,nj->nvi", R, np.asarray(X, dtype=np.float64)) + t[None]
    z = Xc[..., 2]
    zs = np.where(z > near, z, 1.0)
    u = K[None, :, 0] * Xc[..., 0] / zs + K[None, :, 2]
    v = K[None, :, 1] * Xc[..., 1] / zs + K[None, :, 3]
    return (z > near) & (u >= 0) & (u < wh[None, :, 0]) & (v >= 0) & (v < wh[None, :, 1])


def scene_files(scene: dict, d: str) -> str:
    for k in SCENE_KEYS:
        np.save(os.path.join(d, k + ".npy"), np.ascontiguousarray(scene[k], dtype=np.float64))
    return d


def _oracle_job(job):
    """One process's share of a sample (runs in a spawned worker): forward
    and backward of its pixels of one view, plus the view's track term when
    given.  Returns the seconds its oracle calls took."""
    scene_dir, cam_args, pix, v, trk = job
    import oracle
    arrs = {k: np.load(os.path.join(scene_dir, k + ".npy"), mmap_mode="r") for k in SCENE_KEYS}
    sc = oracle.Scene(**arrs)
    cam = oracle.camera_from_rt(*cam_args)
    t0 = time.perf_counter()
    if len(pix):
        oracle.render(sc, cam, pixels=pix)
        oracle.render_bwd(sc, cam, v, pixels=pix)
    if trk is not None:
        X, op, xy = trk
        oracle.track(X, op, np.zeros(len(op), np.int32), xy, [cam], 1.0, 0.1)
    return time.perf_counter() - t0


class OraclePool:
    """Spawned worker processes for the oracle (spawn: safe beside a CUDA
    context).  `procs` processes; at most one per host core, fewer when the
    host memory would not hold one oracle working set per process."""

    def __init__(self, n_gaussians: int, procs: int = 0):
        import multiprocessing
        cores = os.cpu_count() or 1
        try:
            mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
        except (ValueError, OSError, AttributeError):
            mem = 64 << 30
        per_proc = 400 * max(n_gaussians, 1) + (256 << 20)   # projected records, sort buffers
        fit = max(1, int(0.4 * mem // per_proc))
        self.procs = max(1, min(procs or cores, cores, fit))
        self.pool = multiprocessing.get_context("spawn").Pool(self.procs)

    def run(self, scene_dir, cam_args, pix, v, trk=None, procs=None):
        """Wall seconds of one sample split over `procs` processes (default
        all); the track term goes to the first share."""
        n = procs or self.procs
        parts = np.array_split(np.arange(len(pix)), n)
        jobs = [(scene_dir, cam_args, pix[p], v[p], trk if i == 0 else None) for i, p in enumerate(parts)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_job, jobs, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def _view0_sample(w, rng, n_pix):
    W, H = int(w["wh"][0][0]), int(w["wh"][0][1])
    pix = np.stack([rng.integers(0, W, n_pix), rng.integers(0, H, n_pix)], 1).astype(np.int32)
    v = rng.normal(size=(n_pix, 3))
    return pix, v


def _view0_track(w, rng):
    tr = w["tracks"]
    sel = tr["obs_view"] == 0
    W = float(w["wh"][0][0])
    return tr["X"], tr["obs_point"][sel], rng.uniform(0, W, (int(sel.sum()), 2))


def _cam0(w):
    return (int(w["wh"][0][0]), int(w["wh"][0][1]), w["K"][0], w["Rt"][0])


def calibrate(pool, w, scene_dir, rng, procs, trk):
    """Wall seconds of a call with no pixel work (`fixed`) and per pixel per
    process (`per_px`): a first call warms the processes (imports, page
    mapping) and is discarded; then one and three pixels per process."""
    cam = _cam0(w)
    pix, v = _view0_sample(w, rng, procs)
    pool.run(scene_dir, cam, pix, v, trk, procs)
    t1 = pool.run(scene_dir, cam, pix, v, trk, procs)
    pix, v = _view0_sample(w, rng, 3 * procs)
    t3 = pool.run(scene_dir, cam, pix, v, trk, procs)
    per_px = max((t3 - t1) / 2.0, 0.02 * t1, 1e-6)
    return max(t1 - per_px, 0.0), per_px


def timed_sample(pool, w, scene_dir, rng, seconds, procs):
    """Pixels per second of the oracle on `procs` processes over random
    pixels of view 0 (plus its track term), the sample sized to about
    `seconds` of wall time.  Returns (px/s, pixels, wall seconds)."""
    trk = _view0_track(w, rng)
    fixed, per_px = calibrate(pool, w, scene_dir, rng, procs, trk)
    n = int(max(1, min(20000, (seconds - fixed) / per_px))) * procs
    pix, v = _view0_sample(w, rng, n)
    t = pool.run(scene_dir, _cam0(w), pix, v, trk, procs)
    return n / t, n, t


def config_timing(pool, name, rng, shrink, seconds):
    """The oracle on one small configuration: all cores over its full frame,
    one core over a pixel sample.  Returns a dict with both rates and the
    cost per evaluated (pixel, visible Gaussian) pair of the all-cores run."""
    import tempfile
    import oracle
    w = synth.make_workload(name, **shrink)
    d = scene_files(w["scene"], tempfile.mkdtemp(prefix="gs_orc_"))
    W, H = int(w["wh"][0][0]), int(w["wh"][0][1])
    cam = _cam0(w)
    pix = np.stack(np.meshgrid(np.arange(W), np.arange(H)), -1).reshape(-1, 2).astype(np.int32)
    v = rng.normal(size=(len(pix), 3))
    t_all = pool.run(d, cam, pix, v)
    proj = oracle.project(oracle.Scene(**w["scene"]), oracle.camera_from_rt(*cam))
    g_v = int((proj[:, oracle.P["visible"]] > 0).sum())
    rate1, n1, t1 = timed_sample(pool, w, d, rng, seconds, 1)
    return dict(view="%dx%d" % (W, H), gaussians=w["workload"].n_gaussians if not shrink.get("n_gaussians")
                else shrink["n_gaussians"], visible=g_v,
                all_cores=dict(value=len(pix) / t_all / 1e6, seconds=t_all, pixels=len(pix)),
                one_core=dict(value=rate1 / 1e6, seconds=t1, pixels=n1),
                s_per_pair=t_all * pool.procs / (len(pix) * max(g_v, 1)))


def cpu_baseline(w, seconds, counts=None):
    """The oracle on the machine's host cores, in the metric's unit:
       value        all cores, a bounded random pixel sample of view 0 of the
                    benchmark workload (forward + backward over all its
                    Gaussians, plus view 0's track term);
       single_core  the same on one process;
       configs      the tiny configuration (full frame) and a reduced mid
                    one (1 view 320x214, 20k Gaussians SH3) measured, and
       extrapolated the benchmark step from the reduced mid configuration's
                    cost per (pixel, visible Gaussian), linear in
                    sum_v P_v G_v (G_v from the GPU step's own counts)."""
    import tempfile
    rng = np.random.default_rng(123)
    pool = OraclePool(w["workload"].n_gaussians)
    try:
        d = scene_files(w["scene"], tempfile.mkdtemp(prefix="gs_orc_"))
        rate, n, t = timed_sample(pool, w, d, rng, seconds, pool.procs)
        rate1, n1, t1 = timed_sample(pool, w, d, rng, seconds / 2, 1)
        cfg = dict(tiny=config_timing(pool, "tiny", rng, {}, 4.0),
                   mid_reduced=config_timing(pool, "mid", rng, dict(n_gaussians=20000, n_views=1, width=(320, 320),
                                                                    height=(214, 214), n_tracks=10), 4.0))
    finally:
        pool.close()
    W, H = int(w["wh"][0][0]), int(w["wh"][0][1])
    out = dict(value=rate / 1e6, unit=UNIT, cores=pool.procs, host_cores=os.cpu_count(), kind="oracle",
               sample="fwd+bwd of %d random pixels of view 0 (%dx%d) over all %d Gaussians + view-0 track "
                      "term, FP64 C oracle, %d processes, %.1f s wall" % (n, W, H, w["workload"].n_gaussians,
                                                                          pool.procs, t),
               single_core=dict(value=rate1 / 1e6, pixels=n1, seconds=t1), configs=cfg)
    if counts and counts.get("pairs_brute"):
        c = cfg["mid_reduced"]["s_per_pair"]
        t_step = c * counts["pairs_brute"] / pool.procs
        out["extrapolated"] = dict(value=counts["pixels"] / t_step / 1e6, unit=UNIT,
                                   basis="extrapolated: %.3g s per (pixel, visible Gaussian) from mid_reduced "
                                         "x %d pairs (sum_v P_v G_v of the step) / %d processes" % (
                                             c, counts["pairs_brute"], pool.procs))
    return out


def run_reference(args, w):
    """The reference arm: the oracle as it stands on the host cores, each
    step a bounded pixel sample of view 0 of the same workload (all cores),
    sized so that the whole run ends within a few minutes."""
    import tempfile
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    rng = np.random.default_rng(0)
    pool = OraclePool(w["workload"].n_gaussians)
    try:
        d = scene_files(w["scene"], tempfile.mkdtemp(prefix="gs_orc_"))
        cam = _cam0(w)
        trk = _view0_track(w, rng)
        # the calibration's three calls are warm-up steps
        fixed, per_px = calibrate(pool, w, d, rng, pool.procs, trk)
        budget = 150.0 / max(args.steps + args.warmup, 1)
        n_pix = pool.procs * int(max(1, min(5000, (budget - fixed) / per_px)))
        for _ in range(max(args.warmup - 3, 0)):
            pix, v = _view0_sample(w, rng, n_pix)
            pool.run(d, cam, pix, v, trk)
        times = []
        for _ in range(args.steps):
            pix, v = _view0_sample(w, rng, n_pix)
            times.append(pool.run(d, cam, pix, v, trk))
    finally:
        pool.close()
    tot = sum(times)
    value = n_pix * args.steps / 1e6 / tot
    sample = ("fwd+bwd of %d random pixels of view 0 over all Gaussians + view-0 track term per step, FP64 C "
              "oracle on %d processes" % (n_pix, pool.procs))
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * tot / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload_desc(args.workload, w), sample="%d pixels of view 0 per step" % n_pix),
                cpu_baseline=dict(value=value, unit=UNIT, cores=pool.procs, kind="oracle", sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.dev = device_id
        self.proc = None
        self.lines = []
        self.t_on = None
        self.t_off = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark_on(self):
        self.t_on = time.time()

    def mark_off(self):
        self.t_off = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l for (t, l) in self.lines if self.t_on is None or (self.t_on <= t <= (self.t_off or t))]
        if not rows:
            rows = [l for _, l in self.lines]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            p = [x.strip() for x in r.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))


def torch_visible(device):
    """visible(X, wh, K, Rt) for synth.tracks, evaluated with torch on the
    device (the pinhole projection of the track points)."""
    import torch

    def visible(X, wh, K, Rt):
        Xt = torch.as_tensor(np.asarray(X), dtype=torch.float64, device=device)
        Rtt = torch.as_tensor(np.asarray(Rt), dtype=torch.float64, device=device)
        Kt = torch.as_tensor(np.asarray(K), dtype=torch.float64, device=device)
        wht = torch.as_tensor(np.asarray(wh), dtype=torch.float64, device=device)
        Xc = torch.einsum("vij,nj->nvi", Rtt[:, :9].reshape(-1, 3, 3), Xt) + Rtt[None, :, 9:]
        z = Xc[..., 2]
        zs = torch.where(z > 0.01, z, torch.ones_like(z))
        u = Kt[None, :, 0] * Xc[..., 0] / zs + Kt[None, :, 2]
        v = Kt[None, :, 1] * Xc[..., 1] / zs + Kt[None, :, 3]
        ok = (z > 0.01) & (u >= 0) & (u < wht[None, :, 0]) & (v >= 0) & (v < wht[None, :, 1])
        return ok.cpu().numpy()
    return visible


def gpu_inputs(name, device, w=None):
    """Synthetic workload on the device.  Targets are renders of the
    ground-truth scene at the ground-truth poses (16 views per launch, one
    batch laid out on the device and reused); track observations are the
    projections of the track points at those poses plus the workload's pixel
    noise (and outliers), drawn over the views that see each point."""
    import torch
    from paper_2603_04847_gb300 import Batch, Cameras, Gaussians, Renderer
    if w is None:
        w = synth.make_workload(name, visible=torch_visible(device))
    wh, K = w["wh"], w["K"]
    V = len(wh)
    cams_gt = Cameras.from_numpy(wh, K, w["Rt_gt"], device=device)
    g_gt = Gaussians.from_numpy(w["gt"], device=device)
    P = (wh[:, 0].astype(np.int64) * wh[:, 1])
    off = np.concatenate([[0], np.cumsum(P)])
    targets = torch.empty((int(off[-1]), 3), dtype=torch.float32, device=device)
    nb = min(16, V)
    b = Batch(cams_gt, list(range(nb)), device=device, capacity=Batch.capacity_for(cams_gt, nb))
    r = Renderer(g_gt.n, cams_gt, b, device=device)
    for v0 in range(0, V, nb):
        views = list(range(v0, min(V, v0 + nb)))
        if len(views) < nb:
            b = Batch(cams_gt, views, device=device)
            r = Renderer(g_gt.n, cams_gt, b, device=device)
        else:
            b.set_views(cams_gt, views)
        r.ensure_capacity(g_gt)
        r.forward(g_gt)
        targets[int(off[v0]):int(off[views[-1] + 1])].copy_(r.image[:b.pixels])
    del r
    tr = w["tracks"]
    X = torch.as_tensor(tr["X"], dtype=torch.float32, device=device)
    Rt = torch.as_tensor(w["Rt_gt"], dtype=torch.float32, device=device)
    Kt = torch.as_tensor(K, dtype=torch.float32, device=device)
    op = torch.as_tensor(tr["obs_point"], dtype=torch.int64, device=device)
    ov = torch.as_tensor(tr["obs_view"], dtype=torch.int64, device=device)
    R = Rt[ov, :9].reshape(-1, 3, 3)
    Xc = torch.einsum("nij,nj->ni", R, X[op]) + Rt[ov, 9:]
    uv = torch.stack([Kt[ov, 0] * Xc[:, 0] / Xc[:, 2] + Kt[ov, 2], Kt[ov, 1] * Xc[:, 1] / Xc[:, 2] + Kt[ov, 3]], 1)
    uv = uv + torch.as_tensor(tr["noise"], dtype=torch.float32, device=device)
    out = torch.as_tensor(tr["outlier"], device=device)
    whv = torch.as_tensor(wh, dtype=torch.float32, device=device)[ov]
    uv = torch.where(out[:, None], torch.as_tensor(tr["outlier_uv01"], dtype=torch.float32, device=device) * whv, uv)
    g = Gaussians.from_numpy(w["scene"], device=device)
    cams = Cameras.from_numpy(wh, K, w["Rt"], device=device)
    return dict(w=w, g=g, cams=cams, X=X.clone(), obs_point=op.to(torch.int32).contiguous(),
                obs_xy=uv.contiguous(), view_obs_offset=torch.as_tensor(tr["view_obs_offset"], device=device),
                targets=targets, off=off)


def uneven(w) -> bool:
    W = w["workload"]
    return W.width[0] != W.width[1] or W.height[0] != W.height[1]


def tuning_trials(tune):
    """Best eager step time (ms) the autotuner measured per tile size, and
    per tile size the forward/backward stage times per staging batch."""
    t = tune.get("timings", {})
    out = {}
    for k, v in t.items():
        tile, what = k.split("/", 1)
        d = out.setdefault(tile, {})
        if what.startswith("step@"):
            d["step_ms"] = min(d.get("step_ms", float("inf")), v)
        else:
            d[what.replace("stages@", "batch")] = {n: round(x, 4) for n, x in v.items()}
    return out


def tune_child(workload, mode, local, cache_path, lambda_ssim=0.0, w_path=None, deterministic=False):
    """Autotunes the step of `workload` on GPU `local` and writes the result
    (with its trial timings) to the tuning cache at cache_path.  w_path: the
    synthetic workload pickled by the parent (saves drawing it again)."""
    import json
    import pickle
    import torch
    torch.cuda.set_device(local)
    from paper_2603_04847_gb300.autotune import autotune
    w = None
    if w_path:
        with open(w_path, "rb") as f:
            w = pickle.load(f)
    inp = gpu_inputs(workload, "cuda:%d" % local, w)
    W = inp["w"]["workload"]
    views = list(range(min(W.batch, W.n_views)))
    js = make_step(inp, views, mode, W.lambda_ba, lambda_ssim=lambda_ssim, dynamic=uneven(inp["w"]),
                   deterministic=deterministic)
    tune = autotune(js, use_cache=True, cache_path=cache_path)
    with open(cache_path) as f:
        cache = json.load(f)
    for k in cache:
        cache[k]["timings_saved"] = tune.get("timings", {})
    with open(cache_path, "w") as f:
        json.dump(cache, f)


def make_step(inp, views, mode, lambda_ba, tile=16, lambda_ssim=0.0, dynamic=False, deterministic=False,
              variant="full"):
    """variant: the paper's ablation variants -- frozen-poses (no pose
    update), photometric-only (lambda_BA = 0: no track term), merged-tracks
    (the track points are Gaussian means: the tracks' point ids index the
    Gaussians)."""
    from paper_2603_04847_gb300 import Hyper, JointStep
    h = Hyper(lambda_ba=0.0 if variant == "photometric-only" else lambda_ba, lambda_ssim=lambda_ssim,
              freeze_poses=variant == "frozen-poses")
    js = JointStep(inp["g"], inp["cams"], inp["X"], inp["obs_point"], inp["obs_xy"], inp["view_obs_offset"],
                   inp["targets"], inp["off"], views, h, mode=mode, tile=tile, dynamic_batch=dynamic,
                   deterministic=deterministic, merged_tracks=variant == "merged-tracks")
    js.ensure_capacity()
    return js


def time_graph(js, steps, flush, use_graph=True, batches=None):
    """Per-step device times (ms).  With `batches` (pinned [steps, B] int32
    view ids), each timed step first copies its view ids to the device."""
    import torch
    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(st)
        if batches is not None:
            set_views_async(js, batches[i])
        js.run() if use_graph else js.step()
        evs[i][1].record(st)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def set_views_async(js, views_pinned):
    """Device copy of a batch's view ids, no host sync: views of the same
    per-slot sizes, or any views of a batch laid out on the device (the
    step recomputes its offsets).  The host copies of the layout follow."""
    js.batch.views.copy_(views_pinned, non_blocking=True)
    vs = views_pinned.numpy().astype(np.int64)
    js.batch._set_host(js.cams, vs)
    if js.mode != "batched":
        for b, sb in enumerate(js.slot_batches):
            sb.views.copy_(views_pinned[b:b + 1], non_blocking=True)
            sb._set_host(js.cams, vs[b:b + 1])
    js.views = vs


def batch_pixels(cams, views) -> int:
    wh = cams.wh_host[np.asarray(views, dtype=np.int64).reshape(-1)]
    return int((wh[:, 0] * wh[:, 1]).sum())


def stage_times(js, reps, flush):
    """Per-stage device times (ms, mean over reps) of the eager step, with
    CUDA events recorded on the launching stream between stages."""
    import torch
    st = torch.cuda.current_stream()
    acc = {}
    for _ in range(reps):
        flush.zero_()
        marks = [("start", torch.cuda.Event(enable_timing=True))]
        marks[0][1].record(st)

        def mark(name):
            e = torch.cuda.Event(enable_timing=True)
            e.record(st)
            marks.append((name, e))
        js.step(mark)
        torch.cuda.synchronize()
        for (n0, e0), (n1, e1) in zip(marks[:-1], marks[1:]):
            acc[n1] = acc.get(n1, 0.0) + e0.elapsed_time(e1)
    return {k: v / reps for k, v in acc.items()}


# stage -> committed ncu summary holding that kernel's DRAM bytes per launch
NCU_SUMMARY = {"raster_bwd": "render_bwd_mid_8x1237x822_200k.md"}


def ncu_traffic(stage, workload, js, model_bytes=None):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of the stage's
    kernel, from its committed ncu summary -- only while the kernel source
    and the staging batch are those the capture was taken on (else None:
    the counters no longer describe this kernel).  A capture of a smaller
    workload of the same kernel is scaled to this launch by the ratio of
    the algorithmic bytes (model_bytes, this launch) to those of the
    captured launch; the result says so."""
    import hashlib
    from paper_2603_04847_gb300.core import gs_get_tuning
    name = NCU_SUMMARY.get(stage)
    if name is None or getattr(js, "deterministic", False):
        return None   # no capture of this stage, or another instantiation of its kernel
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            kv = dict(line.strip().split(": ", 1) for line in f if ": " in line and line.startswith("    "))
        with open(os.path.join(ROOT, kv["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, KeyError, ValueError):
        return None
    if sha != kv.get("source_sha256"):
        return None
    if str(gs_get_tuning()["render_bwd_batch"]) != kv.get("render_bwd_batch") or str(js.tile) != kv.get("tile"):
        return None
    t = int(kv["traffic_bytes_per_launch"])
    if workload == kv.get("workload"):
        return t
    if model_bytes is None or "algorithmic_bytes_per_launch" not in kv:
        return None
    return dict(bytes=int(t * model_bytes / int(kv["algorithmic_bytes_per_launch"])),
                scaled_from="%s capture (%d bytes per launch, algorithmic %s), x algorithmic bytes ratio" % (
                    kv.get("workload"), t, kv["algorithmic_bytes_per_launch"]))


def algorithmic_model(js):
    """Algorithmic bytes per stage (each intermediate written once and read
    once; the sort as one read + one write of its 12-byte pairs) and the
    compositing pair counts, from this step's own device counters."""
    import torch
    g = js.g
    N = g.n
    K = g.sh.shape[1]
    B = js.batch.B
    P = js.batch.pixels
    I = sum(rr.n_instances() for rr in js.renderers)
    vis_slot = [(rr.proj.n_tiles[:N * rr.batch.B].reshape(rr.batch.B, N) > 0).sum(1).cpu().numpy()
                for rr in js.renderers]
    vis = int(sum(int(v.sum()) for v in vis_slot))
    # brute-force pairs sum_v P_v G_v (the oracle's per-pixel loop)
    pairs_brute = int(sum(int((np.diff(rr.batch.px_offset_host) * v).sum())
                          for rr, v in zip(js.renderers, vis_slot)))
    pairs_bwd = sum(int(rr.n_contrib[:rr.batch.pixels].to(torch.int64).sum().item()) for rr in js.renderers)
    added = sum(rr.count_added(js.g, js.Rt) for rr in js.renderers)
    n_tiles_total = sum(int(rr.batch.tile_offset_host[-1]) for rr in js.renderers)
    pbytes = N * (44 + 12 * K)
    M_b = int(sum(int(js.view_obs_offset[v + 1] - js.view_obs_offset[v]) for v in js.views))
    model = {
        "project": pbytes + vis * 60 + (B * N - vis) * 4,
        "sort": B * N * 12 + vis * 20 + I * 24 + I * 8 + n_tiles_total * 8,
        "render_fwd": I * 40 + P * 20,
        "raster_bwd": I * 40 + P * 32 + vis * 36,
        "project_bwd": pbytes + vis * 36 + B * N * 4 + 2 * pbytes,
        "track": M_b * 24 + min(M_b, js.X.shape[0]) * 24,
        "adam": (N * (7 + 4 + 3 * K) + js.X.shape[0] * 3) * 4 * 7,
    }
    return model, dict(instances=I, visible_records=vis, pairs_bwd=pairs_bwd, added=added, pixels=P,
                       obs_in_batch=M_b, pairs_brute=pairs_brute)


def slowest_rank_time(local_time: float, device="cpu") -> float:
    """Whole-job time of a replica run (any unit): every rank's timed region
    ends at a barrier and the job took as long as its slowest rank (MAX over
    ranks).  With no process group (one rank) it is the local time.  Works
    on any backend (NCCL with a CUDA device, gloo on the CPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_time)
    t = torch.tensor([float(local_time)], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def spread(xs):
    """median, p10, p90 of a list of numbers."""
    a = np.asarray(xs, dtype=np.float64)
    return dict(median=float(np.median(a)), p10=float(np.percentile(a, 10)), p90=float(np.percentile(a, 90)))


def run_ours(args):
    import pickle
    import tempfile
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    from paper_2603_04847_gb300 import build as libbuild
    libbuild.build()
    w = synth.make_workload(args.workload, visible=torch_visible(dev))
    tune_cache = None
    if not args.profile_steps:
        # tune in a child process, which writes the tuning cache this process
        # then reads: a process that has run the other tile size's kernels
        # measured ~2 % slower with the chosen one
        import multiprocessing
        tdir = tempfile.mkdtemp(prefix="gs_tune_")
        tune_cache = os.path.join(tdir, "autotune.json")
        w_path = os.path.join(tdir, "workload.pkl")
        with open(w_path, "wb") as f:
            pickle.dump(w, f, protocol=4)
        child = multiprocessing.get_context("spawn").Process(
            target=tune_child, args=(args.workload, args.mode, local, tune_cache, args.lambda_ssim, w_path,
                                     args.deterministic))
        child.start()
        child.join()
        if child.exitcode != 0:
            raise RuntimeError("autotuning process failed (exit code %s)" % child.exitcode)
    inp = gpu_inputs(args.workload, dev, w)
    W = w["workload"]
    dyn = uneven(w)
    views = list(range(min(W.batch, W.n_views)))
    js = make_step(inp, views, args.mode, W.lambda_ba, lambda_ssim=args.lambda_ssim, dynamic=dyn,
                   deterministic=args.deterministic, variant=args.variant)
    # random batches (Algorithm 1, "Sample image indices") when the workload
    # has more views than one batch
    n_batches = args.warmup + args.steps + max(10, args.steps) + 8
    rng = np.random.default_rng(1234)
    batch_list = None
    if W.n_views > W.batch:
        batch_list = torch.tensor(np.stack(synth.batches(rng, W.n_views, W.batch, n_batches)).astype(np.int32)
                                  ).pin_memory()
    if args.profile_steps:
        if batch_list is not None:
            set_views_async(js, batch_list[0])
        js.ensure_capacity()
        for _ in range(args.profile_steps):
            js.step()
        torch.cuda.synchronize()
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    from paper_2603_04847_gb300.autotune import autotune
    tune = autotune(js, use_cache=True, cache_path=tune_cache)
    if not tune.get("cached"):
        raise RuntimeError("the tuning cache written by the tuning process was not found")
    tune["timings"] = tune.get("timings_saved", {})
    js.ensure_capacity()
    use_graph = not args.no_graph
    if batch_list is not None:
        # every batch has its own instance count: size the instance buffers
        # for the largest of all batches this run will use (with headroom)
        # before capturing, so no timed step can overflow them
        for i in range(len(batch_list)):
            set_views_async(js, batch_list[i])
            js.ensure_capacity()
        set_views_async(js, batch_list[0])
    if use_graph:
        js.capture(warmup=1)
    bcur = 0
    for _ in range(args.warmup):
        flush.zero_()
        if batch_list is not None:
            set_views_async(js, batch_list[bcur])
            bcur += 1
        js.run() if use_graph else js.step()
    torch.cuda.synchronize()
    flags = js.status_flags()
    if flags:
        raise RuntimeError("device status flags %d after warm-up" % flags)

    t_start = bcur
    timed_batches = None if batch_list is None else batch_list[bcur:bcur + args.steps]
    px_steps = ([js.batch.pixels] * args.steps if timed_batches is None else
                [batch_pixels(js.cams, timed_batches[i].numpy()) for i in range(args.steps)])
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_on()
    times = time_graph(js, args.steps, flush, use_graph, timed_batches)
    torch.cuda.synchronize()
    clocks.mark_off()
    tot = slowest_rank_time(sum(times), dev)   # ms, as time_graph returns
    clk = clocks.stop()
    if js.status_flags():
        raise RuntimeError("device status flags %d during the timed steps" % js.status_flags())
    ms = tot / args.steps
    P_mean = sum(px_steps) / len(px_steps)
    value = ws * sum(px_steps) / 1e6 / (tot / 1e3)
    per_step = dict(ms=spread(times), value=spread([p / 1e6 / (t / 1e3) for p, t in zip(px_steps, times)]))

    # per-stage event timing of the same step (eager), for the roofline
    st_ms = stage_times(js, 5, flush)
    model, counts = algorithmic_model(js)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    stages = {k: dict(ms=st_ms.get(k, 0.0)) for k in list(model) + [k for k in st_ms if k not in model]}
    for k in stages:
        t = stages[k]["ms"]
        if k in model and t > 0:
            stages[k]["GBps"] = model[k] / (t * 1e-3) / 1e9
            stages[k]["hbm_frac"] = stages[k]["GBps"] / hbm_peak
    # the dominant kernel: the longest single-kernel stage (the sort stage
    # is a dozen kernels, none of them near the top of the launch list; its
    # HBM fraction is in `stages`).  The step clears the backward's
    # screen-space records on the side stream, so the raster_bwd stage is
    # the compositing backward's launch alone
    kern_ms = dict(st_ms)
    dominant = max(("project", "render_fwd", "raster_bwd", "project_bwd"), key=lambda k: kern_ms.get(k, 0))
    # the compositing kernels are bound by FP32/SFU issue, not HBM: report
    # their pair throughput against the FP32 lane peak
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = sms * 128 * 2 * (peaks.get("sm_max_mhz", 2070.0) * 1e6) / 1e12   # TFLOP/s, FMA = 2
    # Algorithmic flops of compositing (FMA = 2): every examined position
    # (sum of n_contrib) costs the alpha test, 10 flops (exponent 8, exp 1,
    # clamp 1); every composited splat (sum of n_added) costs 9 more in the
    # forward (transmittance 2, weight 1, colour 6) and 60 more in the
    # backward (transmittance and reciprocal 3, colour gradient 6,
    # alpha gradient 15, colour-behind update 6, conic/mean/opacity
    # gradients 30).
    ALU = {"render_fwd": (10.0, 9.0), "raster_bwd": (10.0, 60.0)}
    traffic = ncu_traffic(dominant, args.workload, js, model.get(dominant))
    traffic_note = None
    if isinstance(traffic, dict):
        traffic, traffic_note = traffic["bytes"], traffic["scaled_from"]
    kname = {"raster_bwd": "render_bwd_kernel", "render_fwd": "render_fwd_kernel", "project": "project_fwd_kernel",
             "project_bwd": "project_bwd_kernel"}[dominant]
    if dominant in ALU:
        per_pos, per_add = ALU[dominant]
        fl = counts["pairs_bwd"] * per_pos + counts["added"] * per_add
        ach = fl / (kern_ms[dominant] * 1e-3) / 1e12
        roof = dict(kernel=kname, stage=dominant, bound="alu", achieved=ach, peak=fp32_peak, unit="TFLOP/s",
                    frac=ach / fp32_peak, traffic=traffic, launch_ms=kern_ms[dominant],
                    peak_source="derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (
                        sms, peaks.get("sm_max_mhz", 2070.0)),
                    work="%d examined positions x %.0f + %d composited splats x %.0f flop" % (
                        counts["pairs_bwd"], per_pos, counts["added"], per_add))
    else:
        ach = model[dominant] / (kern_ms[dominant] * 1e-3) / 1e9
        roof = dict(kernel=kname, stage=dominant, bound="hbm", achieved=ach, peak=hbm_peak, unit="GB/s",
                    frac=ach / hbm_peak, traffic=traffic, launch_ms=kern_ms[dominant], peak_source=peak_src)
    if traffic_note:
        roof["traffic_note"] = traffic_note

    step_bytes = sum(model.values())
    step_ms_now = sum(v for k, v in st_ms.items())
    # the stricter "compulsory" count: without the compositing kernels'
    # gathers of the staged records (I x 40 bytes each in the forward and the
    # backward), which could stay in L2
    comp_bytes = step_bytes - 2 * 40 * counts["instances"]
    hbm_step = dict(algorithmic_bytes=step_bytes, GBps=step_bytes / (ms * 1e-3) / 1e9,
                    frac=step_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                    compulsory_bytes=comp_bytes, compulsory_frac=comp_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                    note="bytes of the stage-timed batch over the mean graph-replay step time; compulsory: "
                         "without the two I x 40-byte record gathers of the compositing kernels")
    # the compositing stages against the FP32 lane peak as well (their bound)
    for k in ALU:
        if k in stages and kern_ms.get(k, 0) > 0:
            pp, pa = ALU[k]
            tf = (counts["pairs_bwd"] * pp + counts["added"] * pa) / (kern_ms[k] * 1e-3) / 1e12
            stages[k]["TFLOPs"] = tf
            stages[k]["alu_frac"] = tf / fp32_peak

    # plain one-view-per-launch form on the same inputs (eager, no graph)
    plain = None
    if not args.no_plain and args.mode == "batched":
        jp = make_step(inp, views, "plain", W.lambda_ba, tile=js.tile, lambda_ssim=args.lambda_ssim, dynamic=dyn,
                       deterministic=args.deterministic, variant=args.variant)
        npl = max(3, min(args.steps, 10))
        pb = None if batch_list is None else batch_list[:npl]
        if pb is not None:
            for i in range(npl):
                set_views_async(jp, pb[i])
                jp.ensure_capacity()
        for i in range(2):
            flush.zero_()
            if pb is not None:
                set_views_async(jp, pb[i])
            jp.step()
        pt = time_graph(jp, npl, flush, False, pb)
        ppx = [js.batch.pixels] * npl if pb is None else [batch_pixels(js.cams, pb[i].numpy()) for i in range(npl)]
        pms = sum(pt) / len(pt)
        plain = dict(ms_per_step=pms, value=sum(ppx) / 1e6 / (sum(pt) / 1e3), launches_per_step=jp.kernels_per_step(),
                     ms=spread(pt))
        del jp

    # end to end through the public API: every step's target images come
    # from pinned host memory (TargetStream: uploaded one step ahead on a
    # copy stream, overlapping the step before), then the step runs, then
    # its loss is read back; all of it inside the timed region
    from paper_2603_04847_gb300.step import TargetStream
    host_tgt = inp["targets"].cpu().pin_memory()
    ts = TargetStream(js, host_tgt, inp["off"])
    if use_graph:
        js.capture()
    # each step's loss is read back one step later (two pinned buffers and
    # events), so the host enqueues step i + 1 before it waits for step i
    loss_host = [torch.zeros(2, dtype=torch.float64).pin_memory() for _ in range(2)]
    loss_ready = [torch.cuda.Event(), torch.cuda.Event()]
    losses = []
    n_e2e = max(10, args.steps)
    # the same batches as the device-timed steps (after one untimed step on
    # the batch before them), so that the two numbers compare like for like
    plan = []
    for i in range(n_e2e + 1):
        plan.append(None if batch_list is None else batch_list[(t_start - 1 + i) % len(batch_list)])
    # one untimed pass first: the first replay of a freshly captured graph
    # also uploads it to the device
    ts.put(js.views if plan[0] is None else plan[0].numpy())
    ts.begin()
    if plan[0] is not None:
        set_views_async(js, plan[0])
    js.run() if use_graph else js.step()
    ts.end()
    torch.cuda.synchronize()
    plan = plan[1:]
    e2e_px = sum(js.batch.pixels if p is None else batch_pixels(js.cams, p.numpy()) for p in plan[:n_e2e])
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = ts.put(js.views if plan[0] is None else plan[0].numpy())
    h2d_total = h2d
    for i in range(n_e2e):
        ts.begin()
        if plan[i] is not None:
            set_views_async(js, plan[i])
        js.run() if use_graph else js.step()
        ts.end()
        loss_host[i % 2].copy_(js.loss, non_blocking=True)
        loss_ready[i % 2].record()
        if i >= 1:   # the previous step's loss, read on the host
            loss_ready[(i - 1) % 2].synchronize()
            losses.append(float(loss_host[(i - 1) % 2][0]))
        if i + 1 < n_e2e:
            h2d_total += ts.put(js.views if plan[i + 1] is None else plan[i + 1].numpy())
    loss_ready[(n_e2e - 1) % 2].synchronize()
    losses.append(float(loss_host[(n_e2e - 1) % 2][0]))
    torch.cuda.current_stream().synchronize()
    e2e_s = slowest_rank_time(time.perf_counter() - t0, dev)
    if len(losses) != n_e2e or not all(np.isfinite(losses)):
        raise RuntimeError("end-to-end loop: losses not read back for every step")
    if js.status_flags():
        raise RuntimeError("device status flags %d during the end-to-end steps" % js.status_flags())
    h2d_step = h2d_total / n_e2e + 8 * len(inp["off"]) + (4 * W.batch if batch_list is not None else 0)
    e2e = dict(value=ws * e2e_px / 1e6 / e2e_s, unit=UNIT, h2d_bytes_per_step=int(h2d_step),
               d2h_bytes_per_step=16, ms_per_step=e2e_s * 1e3 / n_e2e,
               pipeline="targets uploaded one step ahead on a copy stream (pinned host -> HBM); each step's "
                        "loss read back by the host one step later",
               l2="no flush inside the pipelined loop; the step's working set is larger than L2")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cpu = cpu_baseline(w, args.cpu_seconds, counts)

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
                    ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                    data="synthetic",
                    config=dict(workload_desc(args.workload, w), mode=args.mode,
                                batches="random %d of %d views per step%s" % (
                                    W.batch, W.n_views, ", uneven sizes, laid out on the device" if dyn else "")
                                if batch_list is not None else "all views every step",
                                mean_pixels_per_step=P_mean,
                                variant=args.variant,
                                lambda_ssim=args.lambda_ssim,
                                backward="deterministic (per-instance slots, fixed-order sums)"
                                if args.deterministic else "atomic (per-tile sums added by FP32 atomics)",
                                graph=use_graph, l2="flushed between steps (256 MB write)",
                                tuning=dict(tile=tune["tile"], render_fwd_batch=tune["render_fwd_batch"],
                                            render_bwd_batch=tune["render_bwd_batch"],
                                            sort_blocks_per_sm=tune["sort_blocks_per_sm"],
                                            trials=tuning_trials(tune)),
                                parallelism="replicas" if ws > 1 else "single GPU"),
                    steps_per_s=1e3 / ms, per_step=per_step, e2e=e2e,
                    gpu_launches=js.kernels_per_step() * args.steps,
                    roofline=roof, hbm_step=hbm_step, stages=stages, counts=counts, clocks=clk,
                    cpu_baseline=cpu, plain=plain)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_sfm_ba(args):
    """LM iterations/s of the bundle adjustment of Eq. 4 on a synthetic
    problem shaped like the joint step's tracks: 50 cameras (1000x750) on a
    radius-4 sphere, 20k points in [-1,1]^3 seen by 2-12 cameras each,
    0.5 px noise, 2 % outliers, poses and points perturbed.  The timed
    iterations replay one CUDA graph of the device-side LM iteration; the
    per-stage device times come from one more, host-decided iteration."""
    import torch
    import synth
    from paper_2603_04847_gb300 import Cameras, build as libbuild
    from paper_2603_04847_gb300.ba import BundleAdjuster
    from paper_2603_04847_gb300.core import sfm_ba_objective
    libbuild.build()
    rng = np.random.default_rng(0)
    V, P, W, H = 50, 20000, 1000, 750
    wh, K, Rt = synth.cameras_sphere(rng, V, (W, W), (H, H))
    X = rng.uniform(-1, 1, (P, 3))
    tr = synth.tracks(rng, X, P, (2, 12), V, 0.5, 0.02)
    op, oc = tr["obs_point"], tr["obs_view"]
    R, t = Rt[oc, :9].reshape(-1, 3, 3), Rt[oc, 9:]
    xc = np.einsum("mab,mb->ma", R, X[op]) + t
    xy = np.stack([K[oc, 0] * xc[:, 0] / xc[:, 2] + K[oc, 2], K[oc, 1] * xc[:, 1] / xc[:, 2] + K[oc, 3]], 1)
    xy = xy + tr["noise"]
    out = tr["outlier"]
    xy[out] = tr["outlier_uv01"][out] * [W, H]
    d = rng.normal(0, 0.002, (V, 6))
    d[0] = 0.0
    Rt0 = Rt.copy()
    for i in range(1, V):   # rotate by Rodrigues(phi) and shift by rho (a small perturbation)
        phi, rho = d[i, 3:], d[i, :3]
        th = np.linalg.norm(phi)
        Wx = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
        E = np.eye(3) + np.sin(th) / th * Wx + (1 - np.cos(th)) / th ** 2 * Wx @ Wx
        Rt0[i, :9] = (E @ Rt[i, :9].reshape(3, 3)).reshape(-1)
        Rt0[i, 9:] = E @ Rt[i, 9:] + rho
    cams = Cameras.from_numpy(wh, K, Rt0)
    Xd = torch.as_tensor(X + rng.normal(0, 0.005, X.shape), dtype=torch.float32, device="cuda")
    adj = BundleAdjuster(cams, Xd, op, oc, xy, delta=1.0, lam=1e-4)
    # the robust objective at the true poses and points: a converged LM
    # ends below it (the optimum also fits part of the pixel noise)
    truth = torch.zeros(1, dtype=torch.float64, device="cuda")
    sfm_ba_objective(torch.as_tensor(X, dtype=torch.float32, device="cuda"), Cameras.from_numpy(wh, K, Rt),
                     adj.obs_point, adj.obs_cam, adj.obs_xy, 1.0, truth)
    L_start = adj.objective
    # each iteration: the LM step with the accept / reject on the device,
    # replayed from one CUDA graph (nothing is read back until the end)
    adj.run_graph(args.warmup)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    L0 = adj.objective
    acc0 = adj.accepted()
    t0 = time.perf_counter()
    a.record(st)
    for _ in range(args.steps):
        adj.graph.replay()
    b.record(st)
    torch.cuda.synchronize()
    dev_ms = a.elapsed_time(b) / args.steps
    adj.objective = float(adj.obj[0].item())   # the end-to-end read of the result
    wall = (time.perf_counter() - t0) / args.steps
    acc = adj.accepted() - acc0
    # per-stage device times of one more iteration (events between stages)
    marks = [("start", torch.cuda.Event(enable_timing=True))]
    marks[0][1].record(st)

    def mark(name):
        e = torch.cuda.Event(enable_timing=True)
        e.record(st)
        marks.append((name, e))

    adj.lam = float(adj.lam_dev.item())
    adj.step(mark)     # the host-decided form, for the per-stage times
    torch.cuda.synchronize()
    stages = {marks[i + 1][0]: marks[i][1].elapsed_time(marks[i + 1][1]) for i in range(len(marks) - 1)}
    line = dict(metric="LM iterations/s of the SfM bundle adjustment (Eq. 4)", value=1e3 / dev_ms,
                unit="iterations/s", n_gpus=1, steps=args.steps, warmup=args.warmup, ms_per_step=dev_ms,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload="sfm-ba: %d cameras %dx%d, %d points, %d observations (2-12 per point)"
                            % (V, W, H, P, len(op))),
                e2e=dict(value=1.0 / wall, unit="iterations/s", ms_per_step=1e3 * wall,
                         note="graph replays launched from the host, the objective read back at the end"),
                loop="LM iteration with the accept / reject on the device (sfm_ba_lm_accept), one CUDA graph",
                stages_ms=stages,
                accepted=acc, objective=dict(start=L_start, after_warmup=L0, end=adj.objective, at_truth=float(truth.item())),
                status=adj.status_flags())
    print(json.dumps(line), flush=True)


def run_mcmc(args):
    """MCMC densification steps/s (Sec. 3.3; Algorithm 1 "Relocate / add
    Gaussians") on the 3M-Gaussian training scene: 5 % of the Gaussians dead
    (opacity below 0.005), n = 2.86M live rows in arrays of the 3M cap.  One
    step = relocation of every dead Gaussian, growth by the cited rule
    min(cap, floor(1.05 n)) - n, the Adam-moment restart of every written row
    and its source, and the opacity-gated noise on all means.  The random
    draws are inputs; the parameters are restored outside the timed events
    before every step, so each step does the same work."""
    import torch
    from paper_2603_04847_gb300 import Gaussians, build as libbuild
    from paper_2603_04847_gb300.core import gs_mcmc_grow, gs_mcmc_noise, gs_mcmc_relocate, gs_mcmc_reset_moments
    libbuild.build()
    cap = 3_000_000
    n = 2_860_000
    rng = np.random.default_rng(0)
    w = synth.make_workload("train", n_gaussians=cap, n_views=2, n_tracks=10)
    sc = {k: v.copy() for k, v in w["scene"].items()}
    dead = rng.choice(n, int(0.05 * n), replace=False)
    sc["opacity_logit"][dead] = rng.uniform(-12.0, -5.5, len(dead))
    sc["opacity_logit"][n:] = -20.0                      # the unused rows up to the cap
    g0 = Gaussians.from_numpy(sc)
    g = Gaussians.from_numpy(sc)
    moments = [(torch.zeros_like(t), torch.zeros_like(t)) for t in g.tensors()]
    n_add = max(0, min(cap, int(1.05 * n)) - n)   # the cited growth rule, 5 % up to the cap
    u_dead = torch.as_tensor(rng.uniform(size=n), dtype=torch.float64, device="cuda")
    u_add = torch.as_tensor(rng.uniform(size=n_add), dtype=torch.float64, device="cuda")
    eta = torch.as_tensor(rng.normal(size=(cap, 3)), dtype=torch.float32, device="cuda")
    src = torch.empty(n, dtype=torch.int32, device="cuda")
    src_add = torch.empty(n_add, dtype=torch.int32, device="cuda")
    n_dead = torch.zeros(1, dtype=torch.int32, device="cuda")
    gl = Gaussians(*[t[:n] for t in g.tensors()])

    def step():
        gs_mcmc_relocate(gl, u_dead, src, n_dead)
        gs_mcmc_reset_moments(cap, src, 0, moments)
        gs_mcmc_grow(g, n, u_add, src_add)
        gs_mcmc_reset_moments(cap, src_add, n, moments)
        gs_mcmc_noise(Gaussians(*[t[:n + n_add] for t in g.tensors()]), eta[:n + n_add], 0.05)

    def restore():
        for a, b in zip(g.tensors(), g0.tensors()):
            a.copy_(b)

    for _ in range(args.warmup):
        restore()
        step()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    times = []
    for _ in range(args.steps):
        restore()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        step()
        b.record(st)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = sum(times) / len(times)
    # per-call device times of one more step (events between the calls)
    restore()
    torch.cuda.synchronize()
    names = ("relocate", "reset_moments_relocated", "grow", "reset_moments_grown", "noise")
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
    calls = (lambda: gs_mcmc_relocate(gl, u_dead, src, n_dead),
             lambda: gs_mcmc_reset_moments(cap, src, 0, moments),
             lambda: gs_mcmc_grow(g, n, u_add, src_add),
             lambda: gs_mcmc_reset_moments(cap, src_add, n, moments),
             lambda: gs_mcmc_noise(Gaussians(*[t[:n + n_add] for t in g.tensors()]), eta[:n + n_add], 0.05))
    evs[0].record(st)
    for c, e in zip(calls, evs[1:]):
        c()
        e.record(st)
    torch.cuda.synchronize()
    stages = {k: evs[i].elapsed_time(evs[i + 1]) for i, k in enumerate(names)}
    nd = int(n_dead.item())
    # algorithmic bytes of one step: relocation reads the opacities three
    # times (scan, apply, reset), writes the cdf/rank/count words and copies
    # 59 floats per dead Gaussian; growth the same scan plus 59 floats per
    # new row; the moment restart zeroes 2 x 59 floats per written row and
    # source; the noise reads 14 floats and writes 3 per Gaussian
    K = 59 * 4
    byt = (n * (4 * 3 + 16) + nd * 2 * K) + (n * (4 * 3 + 16) + n_add * 2 * K) + 2 * (nd + n_add) * 2 * 2 * K + \
          (n + n_add) * 4 * 17
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    # the oracle on the host: the same step on all n rows (about 10 s of
    # numpy work)
    import time as _time
    from oracle import mcmc as omcmc
    ns = n
    ps = {k: np.asarray(v[:ns], np.float64) for k, v in sc.items()}
    ud = rng.uniform(size=ns)
    t0 = _time.perf_counter()
    rel, _ = omcmc.relocate(ps, ud)
    grown, _ = omcmc.grow(rel, rng.uniform(size=omcmc.n_grow(ns, cap)))
    omcmc.noise_means(grown["mean"], grown["log_scale"], grown["quat"], grown["opacity_logit"],
                      rng.normal(size=grown["mean"].shape), 0.05)
    t_cpu = _time.perf_counter() - t0
    line = dict(metric="MCMC densification steps/s (relocate + grow + moment restart + noise)", value=1e3 / ms,
                unit="steps/s", n_gpus=1, steps=args.steps, warmup=args.warmup, ms_per_step=ms,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32 (FP64 scan)", data="synthetic",
                config=dict(workload="mcmc: %d of a %d cap Gaussians SH3, %d dead, %d added per step" % (n, cap, nd,
                                                                                                       n_add)),
                per_step=dict(ms=spread(times)), stages_ms=stages,
                roofline=dict(kernel="whole step", bound="hbm", achieved=byt / (ms * 1e-3) / 1e9, peak=hbm,
                              unit="GB/s", frac=byt / (ms * 1e-3) / 1e9 / hbm, traffic=None,
                              peak_source="measured" if "hbm_gbs" in peaks else "fallback"),
                cpu_baseline=dict(value=(ns / n) / t_cpu, unit="steps/s", cores=1, kind="oracle",
                                  sample="the oracle's relocate + grow + noise of the same %d rows (numpy, FP64, "
                                         "one step): %.2f s" % (ns, t_cpu)))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "sfm-ba":
        run_sfm_ba(args)
        return
    if args.workload == "mcmc":
        run_mcmc(args)
        return
    if args.impl == "reference":
        w = synth.make_workload(args.workload, visible=np_visible)
        run_reference(args, w)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
