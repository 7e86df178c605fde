"""Pins of oracle.joint_step, one iteration of Algorithm 1 composed from the
oracle's pinned pieces: its gradients are the derivative of the iteration's
objective L = sum_views l1_weight mean|I^ - I| + lambda_BA sum rho (central
differences in FP64, poses included through Exp), its first Adam step has
the closed form -lr g / (|g| + eps), and the ablation switches (frozen
poses, lambda_BA = 0, merged tracks) change exactly what they name."""
import numpy as np
import pytest

import oracle
from test_oracle_grad import smooth_camera, smooth_scene

HYPER = dict(lr_mean=1.6e-4, lr_log_scale=5e-3, lr_quat=1e-3, lr_opacity=5e-2, lr_sh=2.5e-3, lr_track=1.6e-4,
             lr_pose=1e-5, beta1=0.9, beta2=0.999, eps=1e-15, scene_extent=1.0, lambda_ba=0.3, huber_delta=1.0,
             l1_weight=0.8, freeze_poses=False)
KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


def _problem(seed=0):
    rng = np.random.default_rng(seed)
    sc = smooth_scene(rng, n=5, sh_degree=1)
    cams = [smooth_camera(rng) for _ in range(2)]
    params = {k: getattr(sc, k).copy() for k in KEYS}
    T0 = np.stack([np.concatenate([np.array(c.R[:]), np.array(c.t[:])]) for c in cams])
    wh = np.array([[c.width, c.height] for c in cams])
    K = np.array([[c.fx, c.fy, c.cx, c.cy] for c in cams])
    targets = {v: rng.uniform(0.0, 1.0, (int(wh[v][1]), int(wh[v][0]), 3)) for v in range(2)}
    X = params["mean"][:3] + rng.normal(0, 0.05, (3, 3))
    obs_point = np.array([0, 1, 2, 0, 2], np.int32)
    obs_view = np.array([0, 0, 0, 1, 1], np.int32)
    xy = np.stack([oracle.project_points(X[k:k + 1], cams[v])[0][0] for k, v in zip(obs_point, obs_view)])
    xy = xy + rng.normal(0, 1.5, xy.shape)       # residuals on both sides of delta
    xi = rng.normal(0, 0.01, (2, 6))
    return params, X, T0, xi, wh, K, targets, obs_point, obs_view, xy


def _objective(params, X, T0, xi, wh, K, targets, obs_point, obs_view, xy, h):
    sc = oracle.Scene(**params)
    Rt = [oracle.pose_update(T0[i:i + 1], xi[i:i + 1].copy(), np.zeros((1, 6)), use_adam=False)[1][0]
          for i in range(2)]
    cams = [oracle.camera_from_rt(int(wh[i][0]), int(wh[i][1]), K[i], Rt[i]) for i in range(2)]
    L = 0.0
    for v in range(2):
        L += oracle.l1_loss_grad(oracle.render(sc, cams[v])["image"], targets[v], h["l1_weight"])[0]
    rho = oracle.track(X, obs_point, obs_view, xy, cams, h["huber_delta"], 1.0)[0]
    return L + h["lambda_ba"] * rho


def test_gradients_are_the_derivative_of_the_iteration_objective():
    pr = _problem()
    params, X, T0, xi, wh, K, targets, obs_point, obs_view, xy = pr
    out = oracle.joint_step(params, X, T0, xi, wh, K, [0, 1], targets, obs_point, obs_view, xy, HYPER, {}, 1)
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in KEYS:
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in params[k].shape)
            pp = {kk: v.copy() for kk, v in params.items()}
            pm = {kk: v.copy() for kk, v in params.items()}
            pp[k][idx] += h
            pm[k][idx] -= h
            fd = (_objective(pp, *pr[1:], HYPER) - _objective(pm, *pr[1:], HYPER)) / (2 * h)
            assert out["grads"][k][idx] == pytest.approx(fd, rel=1e-4, abs=1e-8), (k, idx)
    for i in range(3):
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, c] += h
            Xm[i, c] -= h
            fd = (_objective(params, Xp, *pr[2:], HYPER) - _objective(params, Xm, *pr[2:], HYPER)) / (2 * h)
            assert out["g_X"][i, c] == pytest.approx(fd, rel=1e-4, abs=1e-8)
    # pose: d/dxi = Jl(xi)^T (left tangent)
    for v in range(2):
        g_xi = oracle.pose_update(T0[v:v + 1], xi[v:v + 1].copy(), out["tangent"][v:v + 1], use_adam=False)[0][0]
        for c in range(6):
            xp, xm = xi.copy(), xi.copy()
            xp[v, c] += h
            xm[v, c] -= h
            fd = (_objective(params, X, T0, xp, *pr[4:], HYPER) - _objective(params, X, T0, xm, *pr[4:], HYPER)) / (
                2 * h)
            assert g_xi[c] == pytest.approx(fd, rel=1e-4, abs=1e-8), (v, c)


def test_first_adam_step_closed_form_and_loss_terms():
    pr = _problem(2)
    params, X, T0, xi, wh, K, targets, obs_point, obs_view, xy = pr
    out = oracle.joint_step(params, X, T0, xi, wh, K, [0, 1], targets, obs_point, obs_view, xy, HYPER, {}, 1)
    lrs = dict(mean=HYPER["lr_mean"], log_scale=HYPER["lr_log_scale"], quat=HYPER["lr_quat"],
               opacity_logit=HYPER["lr_opacity"], sh=HYPER["lr_sh"])
    for k in KEYS:
        g = out["grads"][k]
        np.testing.assert_allclose(out["params"][k] - params[k], -lrs[k] * g / (np.abs(g) + HYPER["eps"]),
                                   rtol=1e-9, atol=1e-15)
    assert out["loss_ba"] * HYPER["lambda_ba"] + out["loss_photo"] == pytest.approx(
        _objective(params, X, T0, xi, wh, K, targets, obs_point, obs_view, xy, HYPER), rel=1e-12)


def test_ablation_switches():
    pr = _problem(3)
    params, X, T0, xi, wh, K, targets, obs_point, obs_view, xy = pr
    base = oracle.joint_step(params, X, T0, xi, wh, K, [0, 1], targets, obs_point, obs_view, xy, HYPER, {}, 1)
    # frozen poses: xi unchanged, the gradients of everything else as before
    fr = oracle.joint_step(params, X, T0, xi, wh, K, [0, 1], targets, obs_point, obs_view, xy,
                           dict(HYPER, freeze_poses=True), {}, 1)
    np.testing.assert_array_equal(fr["xi"], xi)
    for k in KEYS:
        np.testing.assert_array_equal(fr["grads"][k], base["grads"][k])
    assert not np.array_equal(base["xi"], xi)
    # photometric only: no track term
    ph = oracle.joint_step(params, X, T0, xi, wh, K, [0, 1], targets, obs_point, obs_view, xy,
                           dict(HYPER, lambda_ba=0.0), {}, 1)
    assert ph["loss_ba"] == 0.0 and not ph["g_X"].any()
    np.testing.assert_array_equal(ph["X"], X)
    # merged tracks: the track points are the means; their gradient adds into the means'
    mg = oracle.joint_step(params, X, T0, xi, wh, K, [0, 1], targets, obs_point, obs_view, xy, HYPER, {}, 1,
                           merged_tracks=True)
    tr = oracle.track(params["mean"], obs_point, obs_view, xy,
                      [oracle.camera_from_rt(int(wh[i][0]), int(wh[i][1]), K[i],
                                             oracle.pose_update(T0[i:i + 1], xi[i:i + 1].copy(), np.zeros((1, 6)),
                                                                use_adam=False)[1][0]) for i in range(2)],
                      HYPER["huber_delta"], HYPER["lambda_ba"])
    np.testing.assert_allclose(mg["grads"]["mean"], ph["grads"]["mean"] + tr[1], rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(mg["X"], mg["params"]["mean"])
