"""Pins of the oracle's hand-derived backward pass: central finite
differences in FP64 on tiny knife-edge-free scenes, closed-form zeros and
the translation gauge identity (no GPU)."""
import math

import numpy as np
import pytest

import oracle
import synth


def smooth_scene(rng, n=6, sh_degree=3, clamp_guard=False):
    """A tiny scene whose splats cover a 24x20 image with moderate alpha, so
    that no evaluated alpha sits near 1/255 or 0.99 and T stays far above
    1e-4; FD steps then never cross a discontinuity."""
    K = (sh_degree + 1) ** 2
    mean = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(3.5, 5.0, n)], 1)
    if clamp_guard:
        mean[0] = [2.4, 0.1, 4.0]  # x/z = 0.6 beyond the guard band 1.3 * 12/30
    log_scale = rng.uniform(-0.2, 0.3, (n, 3))
    quat = rng.normal(size=(n, 4))
    ologit = rng.uniform(-1.2, -0.2, n)
    sh = np.zeros((n, K, 3))
    sh[:, 0] = rng.uniform(-0.8, 0.8, (n, 3))
    if K > 1:
        sh[:, 1:] = rng.normal(0, 0.3, (n, K - 1, 3))
    return oracle.Scene(mean, log_scale, quat, ologit, sh)


def smooth_camera(rng):
    from scipy.spatial.transform import Rotation
    R = Rotation.from_rotvec(rng.normal(0, 0.05, 3)).as_matrix()
    t = rng.normal(0, 0.1, 3)
    return oracle.make_camera(24, 20, 30.0, 31.0, 12.3, 9.8, R, t)


def _loss(sc, cam, w):
    return float((oracle.render(sc, cam)["image"] * w).sum())


def _knife_free(sc, cam, eps=1e-3):
    return not oracle.render(sc, cam, knife_eps=eps)["knife"].any()


@pytest.mark.parametrize("seed,clamp", [(0, False), (1, False), (2, True)])
def test_render_backward_matches_central_differences(seed, clamp):
    rng = np.random.default_rng(seed)
    sc = smooth_scene(rng, clamp_guard=clamp)
    cam = smooth_camera(rng)
    assert _knife_free(sc, cam)
    w = rng.normal(size=(20, 24, 3))
    g = oracle.render_bwd(sc, cam, w)
    h = 1e-6
    for name in ("mean", "log_scale", "quat", "opacity_logit", "sh"):
        arr = getattr(sc, name)
        fd = np.zeros(arr.size)
        flat = arr.reshape(-1)
        for i in range(arr.size):
            old = flat[i]
            flat[i] = old + h
            lp = _loss(sc, cam, w)
            flat[i] = old - h
            lm = _loss(sc, cam, w)
            flat[i] = old
            fd[i] = (lp - lm) / (2 * h)
        an = g[name].reshape(-1)
        scale = max(np.abs(fd).max(), 1e-12)
        assert np.abs(an - fd).max() / scale < 1e-6, name
    # pose tangent: T <- Exp(eps) T
    T0 = np.concatenate([np.array(cam.R[:]), np.array(cam.t[:])])
    fd = np.zeros(6)
    for i in range(6):
        vals = []
        for sgn in (1, -1):
            e = np.zeros(6)
            e[i] = sgn * h
            E = oracle.se3_exp(e)
            R = E[:9].reshape(3, 3) @ T0[:9].reshape(3, 3)
            t = E[:9].reshape(3, 3) @ T0[9:] + E[9:]
            c2 = oracle.make_camera(24, 20, cam.fx, cam.fy, cam.cx, cam.cy, R, t)
            vals.append(_loss(sc, c2, w))
        fd[i] = (vals[0] - vals[1]) / (2 * h)
    assert np.abs(g["tangent"] - fd).max() / np.abs(fd).max() < 1e-6


def test_isotropic_gaussian_has_zero_rotation_gradient():
    rng = np.random.default_rng(3)
    sc = oracle.Scene([[0.1, -0.05, 4.0]], [[0.1] * 3], [rng.normal(size=4)], [-0.5],
                      np.full((1, 1, 3), 0.2))
    cam = oracle.make_camera(24, 20, 30, 30, 12, 10, np.eye(3), [0, 0, 0])
    g = oracle.render_bwd(sc, cam, rng.normal(size=(20, 24, 3)))
    assert np.abs(g["quat"]).max() < 1e-14
    assert np.abs(g["log_scale"]).max() > 1e-6


def test_opacity_gradient_closed_form():
    """One splat, L = sum w * image: dL/d(logit) = sum_px w . c G o (1 - o)
    over covered pixels (no clamp active)."""
    rng = np.random.default_rng(4)
    ol = -0.7
    sc = oracle.Scene([[0.0, 0.0, 4.0]], [[0.0] * 3], [[1, 0, 0, 0]], [ol], np.zeros((1, 1, 3)))
    cam = oracle.make_camera(24, 20, 30, 30, 12, 10, np.eye(3), [0, 0, 0])
    w = rng.normal(size=(20, 24, 3))
    g = oracle.render_bwd(sc, cam, w)
    o = 1 / (1 + math.exp(-ol))
    sig2 = (30.0 * 1.0 / 4.0) ** 2 + 0.3
    v, u = np.mgrid[0:20, 0:24]
    G = np.exp(-0.5 * ((u + 0.5 - 12) ** 2 + (v + 0.5 - 10) ** 2) / sig2)
    assert (o * G >= 1 / 255).all()
    want = (w.sum(-1) * 0.5 * G * o * (1 - o)).sum()
    assert g["opacity_logit"][0] == pytest.approx(want, rel=1e-12)


def test_symmetric_target_gives_zero_mean_gradient():
    """A splat centred on a pixel-symmetric image with a symmetric target:
    the L1 (sub)gradient w.r.t. its 2-D mean is zero."""
    cam = oracle.make_camera(24, 20, 30, 30, 12, 10, np.eye(3), [0, 0, 0])
    sc = oracle.Scene([[0.0, 0.0, 4.0]], [[-0.5] * 3], [[1, 0, 0, 0]], [0.0], np.zeros((1, 1, 3)))
    img = oracle.render(sc, cam)["image"]
    target = np.full_like(img, 0.1)  # symmetric about the image centre
    _, v = oracle.l1_loss_grad(img, target)
    g = oracle.render_bwd(sc, cam, v)
    assert np.abs(g["v2d"][0, :2]).max() < 1e-15
    assert np.abs(g["mean"][0, :2]).max() < 1e-15


def test_photometric_pose_gradient_zero_at_ground_truth():
    """Target rendered at the ground-truth pose with identical Gaussians:
    the L1 subgradient is 0 (sign(0) = 0), so the pose gradient is 0."""
    w = synth.make_workload("tiny", n_gaussians=300)
    sc = oracle.Scene(**w["gt"])
    cam = oracle.camera_from_rt(256, 192, w["K"][0], w["Rt"][0])
    img = oracle.render(sc, cam)["image"]
    _, v = oracle.l1_loss_grad(img, img.copy())
    g = oracle.render_bwd(sc, cam, v)
    assert np.abs(g["tangent"]).max() == 0.0


def test_translation_gauge_identity():
    """Shifting the world by d (means, track points) with t_i <- t_i - R_i d
    leaves L unchanged, so sum dL/dmu + sum dL/dX - sum R_i^T g_rho,i = 0.
    Pins the pose gradient (both losses) against the Gaussian and track
    gradients jointly."""
    rng = np.random.default_rng(7)
    sc = smooth_scene(rng, n=8)
    cams = [smooth_camera(rng) for _ in range(3)]
    Wimg = rng.normal(size=(3, 20, 24, 3))
    sum_mu = np.zeros(3)
    sum_t = np.zeros(3)
    for i, cam in enumerate(cams):
        g = oracle.render_bwd(sc, cam, Wimg[i])
        sum_mu += g["mean"].sum(0)
        R = np.array(cam.R[:]).reshape(3, 3)
        sum_t += R.T @ g["tangent"][:3]
    X = rng.normal(0, 0.3, (10, 3)) + [0, 0, 4]
    op = np.repeat(np.arange(10), 3).astype(np.int32)
    oc = np.tile(np.arange(3), 10).astype(np.int32)
    xy = rng.uniform(0, 24, (30, 2))
    _, gX, tan, _ = oracle.track(X, op, oc, xy, cams, delta=1.0, weight=0.3)
    for i, cam in enumerate(cams):
        R = np.array(cam.R[:]).reshape(3, 3)
        sum_t += R.T @ tan[i, :3]
    total = sum_mu + gX.sum(0) - sum_t
    scale = np.abs(sum_mu).max() + np.abs(gX.sum(0)).max()
    assert np.abs(total).max() < 1e-10 * max(scale, 1.0)
