"""Pins of the oracle's SfM bundle adjustment (Eq. 4, Levenberg-Marquardt
over SE(3) poses and points; no GPU): Jacobians against central
differences, the IRLS gradient against the C oracle's Huber track term, the
Schur-complement solve against the dense one, Exp against the C oracle's,
and convergence on a noiseless problem."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ba

W_IMG, H_IMG, F = 400, 300, 320.0


def _problem(seed, n_cams=4, n_pts=12, pix_noise=0.0, outliers=0):
    rng = np.random.default_rng(seed)
    Rt = np.zeros((n_cams, 12))
    for i in range(n_cams):
        a = 2 * np.pi * i / n_cams + rng.uniform(-0.2, 0.2)
        c = 4.0 * np.array([np.cos(a), np.sin(a), rng.uniform(-0.3, 0.3)])
        R, t = synth.look_at(c)
        Rt[i, :9], Rt[i, 9:] = R.reshape(-1), t
    K = np.tile([F, F, W_IMG / 2, H_IMG / 2], (n_cams, 1))
    X = rng.uniform(-1, 1, (n_pts, 3))
    cams, pts = np.meshgrid(np.arange(n_cams), np.arange(n_pts), indexing="ij")
    obs_cam, obs_point = cams.reshape(-1).astype(np.int32), pts.reshape(-1).astype(np.int32)
    r0, _, _ = ba.residuals(X, Rt, K, obs_point, obs_cam, np.zeros((len(obs_cam), 2)))
    xy = r0 + rng.normal(0, pix_noise, r0.shape) if pix_noise else r0.copy()
    if outliers:
        xy[rng.choice(len(xy), outliers, replace=False)] += rng.uniform(20, 60, (outliers, 2))
    return X, Rt, K, obs_point, obs_cam, xy


def test_huber_weight_is_the_derivative_of_rho():
    s = np.array([0.01, 0.5, 0.99, 1.5, 9.0, 400.0])
    h = 1e-6
    fd = (ba.huber_rho(s + h, 1.0) - ba.huber_rho(s - h, 1.0)) / (2 * h)
    assert np.abs(ba.huber_weight(s, 1.0) - fd).max() < 1e-7
    # continuous at s = delta^2
    assert abs(ba.huber_rho(1.0 + 1e-12, 1.0) - ba.huber_rho(1.0, 1.0)) < 1e-9


def test_exp_matches_the_c_oracle():
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.normal(0, 0.7, 6)
        E = ba.se3_exp(d)
        T = oracle.se3_exp(d)
        assert np.abs(E[:, :3].reshape(-1) - T[:9]).max() < 1e-12
        assert np.abs(E[:, 3] - T[9:]).max() < 1e-12


def test_jacobians_match_central_differences():
    X, Rt, K, op, oc, xy = _problem(1, pix_noise=2.0)
    Jp, JX = ba.jacobians(X, Rt, K, op, oc)
    h = 1e-6
    V, P = Rt.shape[0], X.shape[0]
    for i in range(V):
        for a in range(6):
            dc = np.zeros((V, 6))
            dc[i, a] = h
            Xp, Rp = ba.apply_update(X, Rt, dc, np.zeros_like(X))
            Xm, Rm = ba.apply_update(X, Rt, -dc, np.zeros_like(X))
            fd = (ba.residuals(Xp, Rp, K, op, oc, xy)[0] - ba.residuals(Xm, Rm, K, op, oc, xy)[0]) / (2 * h)
            sel = oc == i
            assert np.abs(fd[sel] - Jp[sel, :, a]).max() <= 1e-5 * max(1.0, np.abs(Jp[sel, :, a]).max())
    for k in range(0, P, 3):
        for a in range(3):
            dp = np.zeros_like(X)
            dp[k, a] = h
            fd = (ba.residuals(X + dp, Rt, K, op, oc, xy)[0] - ba.residuals(X - dp, Rt, K, op, oc, xy)[0]) / (2 * h)
            sel = op == k
            assert np.abs(fd[sel] - JX[sel, :, a]).max() <= 1e-5 * max(1.0, np.abs(JX[sel, :, a]).max())


def test_irls_gradient_matches_the_c_track_oracle():
    """2 sum w J^T r is the gradient of Eq. 4's objective; the C oracle's
    Huber track term (Eq. 6, weight 1) computes the same sum independently."""
    X, Rt, K, op, oc, xy = _problem(2, pix_noise=1.5, outliers=5)
    U, Wb, Vb, gc, gp = ba.normal_equations(X, Rt, K, op, oc, xy, 1.0)
    cams = [oracle.camera_from_rt(W_IMG, H_IMG, K[i], Rt[i]) for i in range(Rt.shape[0])]
    loss, gX, tan, masked = oracle.track(X, op, oc, xy, cams, delta=1.0, weight=1.0)
    assert masked == 0
    assert abs(loss - ba.objective(X, Rt, K, op, oc, xy, 1.0)) <= 1e-10 * loss
    assert np.abs(2 * gp - gX).max() <= 1e-9 * np.abs(gX).max()
    assert np.abs(2 * gc - tan).max() <= 1e-9 * np.abs(tan).max()


@pytest.mark.parametrize("lam", [1e-6, 1e-3, 1.0])
def test_schur_solve_equals_the_dense_solve(lam):
    X, Rt, K, op, oc, xy = _problem(3, n_cams=5, n_pts=15, pix_noise=1.0, outliers=3)
    blocks = ba.normal_equations(X, Rt, K, op, oc, xy, 1.0)
    dc1, dp1 = ba.solve_dense(*blocks, op, oc, lam)
    dc2, dp2 = ba.solve_schur(*blocks, op, oc, lam)
    assert not np.any(dc1[0]) and not np.any(dc2[0])
    scale = max(np.abs(dc1).max(), np.abs(dp1).max())
    assert np.abs(dc1 - dc2).max() <= 1e-8 * scale
    assert np.abs(dp1 - dp2).max() <= 1e-8 * scale


def test_lm_recovers_a_noiseless_problem():
    X, Rt, K, op, oc, xy = _problem(4, n_cams=4, n_pts=20)
    rng = np.random.default_rng(5)
    dc = rng.normal(0, 0.01, (Rt.shape[0], 6))
    dc[0] = 0.0
    X0, Rt0 = ba.apply_update(X, Rt, dc, rng.normal(0, 0.02, X.shape))
    L0 = ba.objective(X0, Rt0, K, op, oc, xy, 1.0)
    Xs, Rts, hist = ba.lm(X0, Rt0, K, op, oc, xy, delta=1.0, iters=40)
    assert L0 > 1.0
    assert hist[-1] < 1e-10 * L0
    assert all(b <= a for a, b in zip(hist[:-1], hist[1:]))
    np.testing.assert_array_equal(Rts[0], Rt0[0])   # the gauge camera never moves


def test_lm_with_outliers_lowers_the_robust_objective():
    X, Rt, K, op, oc, xy = _problem(6, n_cams=4, n_pts=20, pix_noise=0.5, outliers=6)
    rng = np.random.default_rng(7)
    dc = rng.normal(0, 0.005, (Rt.shape[0], 6))
    dc[0] = 0.0
    X0, Rt0 = ba.apply_update(X, Rt, dc, rng.normal(0, 0.01, X.shape))
    _, _, hist = ba.lm(X0, Rt0, K, op, oc, xy, delta=1.0, iters=25)
    # the noise and the outliers' linear Huber part remain: the optimum is
    # at or below the objective at the true parameters, far below the start
    L_true = ba.objective(X, Rt, K, op, oc, xy, 1.0)
    assert hist[0] > 1.2 * L_true
    assert hist[-1] <= L_true
    assert all(b <= a for a, b in zip(hist[:-1], hist[1:]))
