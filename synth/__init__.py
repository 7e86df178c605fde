"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the smoke check and the benchmark.  It
holds none of the method's arithmetic: it only draws random numbers, places
cameras and builds index structures.  Anything that needs the method (track
observations are projections of track points; target images are renders)
is produced by the consumer: by the oracle in tests, by the CUDA path in the
benchmark.

The paper's datasets (MipNeRF360, Tanks and Temples, CO3Dv2, ScanNet) are
not available; these scenes stand in for them.  Recipes:

  tiny      1 camera 256x192 at the identity pose, fx=fy=220, c=(128,96);
            means x,y ~ U[-1,1], z ~ U[3,6]; log-scale ~ N(-3, 0.3);
            quaternion ~ N(0, I4) (unnormalised); opacity logit ~ N(0,1);
            SH degree 0 with colour ~ U(0,1); 200 tracks, one observation
            each, noiseless; target scene = means jittered by N(0, 0.02).
  mid       8 cameras on a sphere of radius 4 looking at the origin, each
            1237x822, fx=fy=0.9 W; 200k Gaussians, SH degree 3; 20k tracks
            with 2..12 observations, pixel noise N(0, 0.5^2); poses
            perturbed by 1 deg about a random axis plus 2 % translation.
  batched   32 views of uneven resolution (W ~ U{640..1600},
            H ~ U{480..1066}), 1M Gaussians SH3, 60k tracks with 2..20 obs.
  train     200 views 1600x1066, 3M Gaussians SH3, 100k tracks 3..30 obs
            with 5 % outliers uniform over the image; batches of 8 views.
  large     1000 views W ~ U{960..1920}, H ~ U{540..1080}, 5M Gaussians
            SH3, 400k tracks 2..40 obs, pose noise U[0.5, 3] deg; batches of
            16 random views.
Track observations are drawn over the views that see the track point (in
the image, positive depth) when the consumer passes its projection as
`visible`; the benchmark and the full-size tests do.
For all scenes but `tiny`: means ~ U[-1,1]^3, log-scale ~
N(ln(0.31 (8/N)^(1/3)), 0.3), SH DC coefficients uniform over the range that
maps to colour U(0,1), higher bands N(0, 0.05^2); the optimised scene is the
ground-truth scene with means jittered by N(0, (0.25 scale)^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

# Range of the degree-0 SH coefficient whose colour (0.5 + Y00 * c) spans
# [0, 1]: Y00 = 1 / (2 sqrt(pi)), so c in [-sqrt(pi), sqrt(pi)].
_DC_HALF_RANGE = math.sqrt(math.pi)


@dataclass
class Workload:
    name: str
    seed: int
    n_gaussians: int
    sh_degree: int
    n_views: int
    width: tuple          # (lo, hi) inclusive
    height: tuple
    batch: int            # views per step
    n_tracks: int
    obs_range: tuple      # observations per track (lo, hi) inclusive
    pix_noise: float = 0.5
    outlier_frac: float = 0.0
    rot_noise_deg: tuple = (1.0, 1.0)
    trans_noise_frac: float = 0.02
    lambda_ba: float = 0.1
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "tiny": Workload("tiny", 0, 2000, 0, 1, (256, 256), (192, 192), 1, 200, (1, 1),
                     pix_noise=0.0, rot_noise_deg=(0.0, 0.0), trans_noise_frac=0.0),
    "mid": Workload("mid", 1, 200_000, 3, 8, (1237, 1237), (822, 822), 8, 20_000, (2, 12)),
    "batched": Workload("batched", 2, 1_000_000, 3, 32, (640, 1600), (480, 1066), 32,
                        60_000, (2, 20)),
    "train": Workload("train", 3, 3_000_000, 3, 200, (1600, 1600), (1066, 1066), 8,
                      100_000, (3, 30), outlier_frac=0.05),
    "large": Workload("large", 4, 5_000_000, 3, 1000, (960, 1920), (540, 1080), 16,
                      400_000, (2, 40), rot_noise_deg=(0.5, 3.0)),
}


def gaussians_cube(rng: np.random.Generator, n: int, sh_degree: int):
    """Means uniform in [-1,1]^3, log-scales around the mean spacing."""
    K = (sh_degree + 1) ** 2
    mean = rng.uniform(-1.0, 1.0, size=(n, 3))
    ls_mu = math.log(0.31 * (8.0 / max(n, 1)) ** (1.0 / 3.0))
    log_scale = rng.normal(ls_mu, 0.3, size=(n, 3))
    quat = rng.normal(0.0, 1.0, size=(n, 4))
    opacity_logit = rng.normal(0.0, 1.0, size=n)
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, size=(n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, K - 1, 3))
    return dict(mean=mean, log_scale=log_scale, quat=quat, opacity_logit=opacity_logit, sh=sh)


def gaussians_tiny(rng: np.random.Generator, n: int):
    mean = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(3, 6, n)], 1)
    log_scale = rng.normal(-3.0, 0.3, size=(n, 3))
    quat = rng.normal(0.0, 1.0, size=(n, 4))
    opacity_logit = rng.normal(0.0, 1.0, size=n)
    sh = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, size=(n, 1, 3))
    return dict(mean=mean, log_scale=log_scale, quat=quat, opacity_logit=opacity_logit, sh=sh)


def look_at(center: np.ndarray, target=np.zeros(3), up=np.array([0.0, 0.0, 1.0])):
    """World-to-camera (R, t) for a camera at `center` looking at `target`,
    x right, y down, z forward."""
    f = target - center
    f = f / np.linalg.norm(f)
    r = np.cross(f, up)
    r = r / np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], 0)
    t = -R @ center
    return R, t


def cameras_sphere(rng: np.random.Generator, n_views: int, width, height, radius=4.0,
                   focal_factor=0.9):
    """Cameras at random directions (elevation within +-60 deg) on a sphere,
    looking at the origin.  Returns wh [V,2] int, K [V,4], Rt [V,12]."""
    W = rng.integers(width[0], width[1] + 1, size=n_views)
    H = rng.integers(height[0], height[1] + 1, size=n_views)
    az = rng.uniform(0.0, 2.0 * math.pi, size=n_views)
    el = rng.uniform(-math.pi / 3.0, math.pi / 3.0, size=n_views)
    Rt = np.zeros((n_views, 12))
    K = np.zeros((n_views, 4))
    for i in range(n_views):
        c = radius * np.array([math.cos(el[i]) * math.cos(az[i]),
                               math.cos(el[i]) * math.sin(az[i]), math.sin(el[i])])
        R, t = look_at(c)
        Rt[i, :9] = R.reshape(-1)
        Rt[i, 9:] = t
        f = focal_factor * W[i]
        K[i] = (f, f, W[i] / 2.0, H[i] / 2.0)
    return np.stack([W, H], 1).astype(np.int32), K, Rt


def perturb_poses(rng: np.random.Generator, Rt: np.ndarray, angle_deg, trans_frac):
    """Left-multiply each pose by a rotation of the given angle (deg, or a
    (lo, hi) range) about a random axis and offset t by trans_frac * |t| in a
    random direction."""
    V = Rt.shape[0]
    lo, hi = (angle_deg, angle_deg) if np.isscalar(angle_deg) else angle_deg
    ang = np.deg2rad(rng.uniform(lo, hi, size=V))
    axis = rng.normal(size=(V, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    dirs = rng.normal(size=(V, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    out = Rt.copy()
    for i in range(V):
        Rn = Rotation.from_rotvec(axis[i] * ang[i]).as_matrix()
        R = Rt[i, :9].reshape(3, 3)
        t = Rt[i, 9:]
        out[i, :9] = (Rn @ R).reshape(-1)
        out[i, 9:] = Rn @ t + trans_frac * np.linalg.norm(t) * dirs[i]
    return out


def tracks(rng: np.random.Generator, gt_means: np.ndarray, n_tracks: int, obs_range,
           n_views: int, pix_noise: float, outlier_frac: float = 0.0, visible=None, chunk: int = 8192):
    """Track points (a random subset of ground-truth means) and their
    observations, bucketed by view (view-CSR).  Each track k draws its count
    m_k ~ U{lo..hi} and observes min(m_k, #eligible) distinct views chosen
    uniformly among its eligible ones: every view, or, when `visible` is
    given, the views where the consumer's projection finds the point in the
    image with positive depth -- visible(X [n,3]) -> bool [n, n_views] is
    called on chunks of track points (this module does no projection).  The
    observation pixel is pi(X) + noise, which the consumer computes; this
    returns the noise, the outlier mask and uniform outlier positions in
    [0,1)^2 (to be scaled by the image size)."""
    n_tracks = min(n_tracks, gt_means.shape[0])
    pick = rng.choice(gt_means.shape[0], size=n_tracks, replace=False)
    X = gt_means[pick].copy()
    lo, hi = obs_range
    m = rng.integers(lo, hi + 1, size=n_tracks)
    m = np.minimum(m, n_views)
    if visible is None:
        pts, views = [], []
        for k in range(n_tracks):
            vs = rng.choice(n_views, size=m[k], replace=False)
            pts.append(np.full(m[k], k))
            views.append(vs)
        obs_point = np.concatenate(pts).astype(np.int32) if pts else np.zeros(0, np.int32)
        obs_view = np.concatenate(views).astype(np.int32) if views else np.zeros(0, np.int32)
    else:
        pts, views = [], []
        for k0 in range(0, n_tracks, chunk):
            k1 = min(n_tracks, k0 + chunk)
            vis = np.asarray(visible(X[k0:k1]), dtype=bool).reshape(k1 - k0, n_views)
            # a uniform random subset of the eligible views: the m_k smallest
            # of independent uniform keys, ineligible views keyed past 1
            keys = rng.random((k1 - k0, n_views)) + np.where(vis, 0.0, 2.0)
            order = np.argsort(keys, axis=1, kind="stable")
            take = np.arange(n_views)[None, :] < np.minimum(m[k0:k1], vis.sum(1))[:, None]
            rows, cols = np.nonzero(take)
            pts.append((k0 + rows).astype(np.int32))
            views.append(order[rows, cols].astype(np.int32))
        obs_point = np.concatenate(pts) if pts else np.zeros(0, np.int32)
        obs_view = np.concatenate(views) if views else np.zeros(0, np.int32)
    order = np.argsort(obs_view, kind="stable")
    obs_point, obs_view = obs_point[order], obs_view[order]
    M = obs_point.shape[0]
    noise = rng.normal(0.0, pix_noise, size=(M, 2)) if pix_noise > 0 else np.zeros((M, 2))
    outlier = rng.uniform(size=M) < outlier_frac
    outlier_uv01 = rng.uniform(size=(M, 2))
    offsets = np.zeros(n_views + 1, dtype=np.int64)
    np.add.at(offsets, obs_view + 1, 1)
    offsets = np.cumsum(offsets)
    return dict(X=X, obs_point=obs_point, obs_view=obs_view, view_obs_offset=offsets,
                noise=noise, outlier=outlier, outlier_uv01=outlier_uv01)


def make_workload(name: str, n_gaussians: int | None = None, n_views: int | None = None,
                  width=None, height=None, n_tracks: int | None = None, seed: int | None = None,
                  visible=None):
    """Build every random input of a named workload (optionally shrunk).
    visible(X, wh, K, Rt) -> bool [n, V], supplied by the consumer, restricts
    each track's observations to the views that see its point (the recipe);
    without it every view is eligible."""
    w = WORKLOADS[name]
    seed = w.seed if seed is None else seed
    rng = np.random.default_rng(seed)
    N = w.n_gaussians if n_gaussians is None else n_gaussians
    V = w.n_views if n_views is None else n_views
    width = w.width if width is None else width
    height = w.height if height is None else height
    T = w.n_tracks if n_tracks is None else n_tracks
    out = dict(workload=w, name=name, seed=seed)
    if name == "tiny":
        gt = gaussians_tiny(rng, N)
        wh = np.array([[width[0], height[0]]] * V, dtype=np.int32)
        K = np.array([[220.0, 220.0, width[0] / 2.0, height[0] / 2.0]] * V)
        Rt = np.zeros((V, 12))
        Rt[:, [0, 4, 8]] = 1.0
        cur = {k: v.copy() for k, v in gt.items()}
        cur["mean"] = gt["mean"] + rng.normal(0.0, 0.02, size=gt["mean"].shape)
        Xs = np.stack([rng.uniform(-1, 1, T), rng.uniform(-1, 1, T), rng.uniform(3, 6, T)], 1)
        tr = dict(X=Xs, obs_point=np.arange(T, dtype=np.int32),
                  obs_view=np.zeros(T, dtype=np.int32),
                  view_obs_offset=np.array([0] + [T] * V, dtype=np.int64),
                  noise=np.zeros((T, 2)), outlier=np.zeros(T, bool),
                  outlier_uv01=np.zeros((T, 2)))
        out.update(gt=gt, scene=cur, wh=wh, K=K, Rt_gt=Rt, Rt=Rt.copy(), tracks=tr)
        return out
    gt = gaussians_cube(rng, N, w.sh_degree)
    wh, K, Rt_gt = cameras_sphere(rng, V, width, height)
    Rt = perturb_poses(rng, Rt_gt, w.rot_noise_deg, w.trans_noise_frac)
    scale = np.exp(gt["log_scale"]).mean(axis=1, keepdims=True)
    cur = {k: v.copy() for k, v in gt.items()}
    cur["mean"] = gt["mean"] + rng.normal(size=gt["mean"].shape) * 0.25 * scale
    vis = None if visible is None else (lambda X: visible(X, wh, K, Rt_gt))
    tr = tracks(rng, gt["mean"], T, w.obs_range, V, w.pix_noise, w.outlier_frac, visible=vis)
    out.update(gt=gt, scene=cur, wh=wh, K=K, Rt_gt=Rt_gt, Rt=Rt, tracks=tr)
    return out


def batches(rng: np.random.Generator, n_views: int, batch: int, n_steps: int):
    """Random view batches (Algorithm 1, 'Sample image indices')."""
    return [np.sort(rng.choice(n_views, size=min(batch, n_views), replace=False))
            for _ in range(n_steps)]
