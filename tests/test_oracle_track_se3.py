"""Pins of the oracle's track term (Eq. 6), SE(3) maps, Adam and SH basis
(no GPU)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cam(rng, W=640, H=480):
    R = Rotation.from_rotvec(rng.normal(0, 0.3, 3)).as_matrix()
    return oracle.make_camera(W, H, 500.0, 510.0, W / 2 + 3, H / 2 - 2, R, rng.normal(0, 0.2, 3) + [0, 0, 4])


def test_noiseless_track_zero_residual():
    rng = np.random.default_rng(0)
    cams = [_cam(rng) for _ in range(4)]
    X = rng.uniform(-1, 1, (50, 3))
    op, oc, xy = [], [], []
    for i, c in enumerate(cams):
        uv, _ = oracle.project_points(X, c)
        op += list(range(50))
        oc += [i] * 50
        xy.append(uv)
    loss, gX, tan, masked = oracle.track(X, op, oc, np.concatenate(xy), cams)
    assert masked == 0
    assert loss < 1e-20 and np.abs(gX).max() < 1e-9 and np.abs(tan).max() < 1e-9


def test_huber_branches_closed_form():
    """Point on the optical axis projects to the principal point; an
    observation at distance r gives rho = r^2 (r <= delta) or
    2 delta r - delta^2 (beyond)."""
    cam = oracle.make_camera(100, 100, 50, 50, 50, 50, np.eye(3), [0, 0, 0])
    for r, want in [(0.5, 0.25), (1.0, 1.0), (3.0, 2 * 3.0 - 1.0), (40.0, 79.0)]:
        loss, *_ = oracle.track([[0, 0, 2.0]], [0], [0], [[50.0 + r, 50.0]], [cam], delta=1.0)
        assert loss == pytest.approx(want, rel=1e-14)
    loss, *_ = oracle.track([[0, 0, 2.0]], [0], [0], [[53.0, 54.0]], [cam], delta=2.0)
    assert loss == pytest.approx(2 * 2.0 * 5.0 - 4.0, rel=1e-14)


def test_huber_gradient_norm_beyond_delta():
    """Beyond delta, |d rho / d r| = 2 delta: with an identity camera at
    Z = fx the image-plane gradient maps 1:1 onto dL/dX_x, dL/dX_y."""
    cam = oracle.make_camera(100, 100, 2.0, 2.0, 50, 50, np.eye(3), [0, 0, 0])
    _, gX, _, _ = oracle.track([[0, 0, 2.0]], [0], [0], [[53.0, 46.0]], [cam], delta=1.0, weight=1.0)
    assert math.hypot(gX[0, 0], gX[0, 1]) == pytest.approx(2.0, rel=1e-12)


def test_points_behind_camera_are_masked():
    cam = oracle.make_camera(100, 100, 50, 50, 50, 50, np.eye(3), [0, 0, 0])
    loss, gX, tan, masked = oracle.track([[0, 0, -1.0], [0, 0, 0.001]], [0, 1], [0, 0],
                                         [[1, 1], [2, 2]], [cam])
    assert masked == 2 and loss == 0 and not gX.any() and not tan.any()


def test_track_gradients_central_differences():
    rng = np.random.default_rng(1)
    cams = [_cam(rng) for _ in range(3)]
    X = rng.uniform(-1, 1, (12, 3))
    op = np.repeat(np.arange(12), 3)
    oc = np.tile(np.arange(3), 12)
    xy = []
    for k, i in zip(op, oc):
        uv, _ = oracle.project_points(X[k:k + 1], cams[i])
        xy.append(uv[0] + rng.normal(0, 1.5, 2))  # both Huber branches
    xy = np.array(xy)
    wgt = 0.37
    loss, gX, tan, _ = oracle.track(X, op, oc, xy, cams, weight=wgt)
    h = 1e-6

    def L(Xv, cs):
        return wgt * oracle.track(Xv, op, oc, xy, cs)[0]

    fd = np.zeros_like(X)
    for idx in np.ndindex(X.shape):
        Xp, Xm = X.copy(), X.copy()
        Xp[idx] += h
        Xm[idx] -= h
        fd[idx] = (L(Xp, cams) - L(Xm, cams)) / (2 * h)
    assert np.abs(fd - gX).max() / np.abs(fd).max() < 1e-6
    for i in range(3):
        for a in range(6):
            vals = []
            for sgn in (1, -1):
                e = np.zeros(6)
                e[a] = sgn * h
                E = oracle.se3_exp(e)
                c = cams[i]
                R0 = np.array(c.R[:]).reshape(3, 3)
                t0 = np.array(c.t[:])
                Re = E[:9].reshape(3, 3)
                cs = list(cams)
                cs[i] = oracle.make_camera(c.width, c.height, c.fx, c.fy, c.cx, c.cy, Re @ R0, Re @ t0 + E[9:])
                vals.append(L(X, cs))
            fdv = (vals[0] - vals[1]) / (2 * h)
            assert fdv == pytest.approx(tan[i, a], rel=1e-5, abs=1e-6 * np.abs(tan).max())


def test_se3_exp_matches_scipy_and_log_roundtrip():
    rng = np.random.default_rng(2)
    for _ in range(20):
        axis = rng.normal(size=3)
        phi = axis / np.linalg.norm(axis) * rng.uniform(0.0, 3.0)  # |phi| < pi: Log is unique
        xi = np.concatenate([rng.normal(0, 1, 3), phi])
        T = oracle.se3_exp(xi)
        Rs = Rotation.from_rotvec(xi[3:]).as_matrix()
        np.testing.assert_allclose(T[:9].reshape(3, 3), Rs, atol=1e-13)
        np.testing.assert_allclose(oracle.se3_log(T), xi, atol=1e-10)
    # tiny angles use the series branch
    xi = np.array([0.3, -0.2, 0.1, 1e-7, -2e-7, 5e-8])
    np.testing.assert_allclose(oracle.se3_log(oracle.se3_exp(xi)), xi, atol=1e-14)
    # pure translation: Exp is a translation by rho
    T = oracle.se3_exp([1, 2, 3, 0, 0, 0])
    np.testing.assert_allclose(T, [1, 0, 0, 0, 1, 0, 0, 0, 1, 1, 2, 3], atol=0)


def _compose(A, B):
    Ra, ta = A[:9].reshape(3, 3), A[9:]
    Rb, tb = B[:9].reshape(3, 3), B[9:]
    return np.concatenate([(Ra @ Rb).reshape(-1), Ra @ tb + ta])


def _inverse(A):
    R, t = A[:9].reshape(3, 3), A[9:]
    return np.concatenate([R.T.reshape(-1), -R.T @ t])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_left_jacobian_matches_fd_of_exp(seed):
    """Exp(xi + h e) Exp(xi)^-1 = Exp(Jl(xi) h e) + O(h^2)."""
    rng = np.random.default_rng(seed)
    xi = np.concatenate([rng.normal(0, 1, 3), rng.normal(0, 1.0 if seed else 1e-4, 3)])
    J = oracle.se3_left_jacobian(xi)
    Ti = _inverse(oracle.se3_exp(xi))
    h = 1e-6
    fd = np.zeros((6, 6))
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        lp = oracle.se3_log(_compose(oracle.se3_exp(xi + e), Ti))
        lm = oracle.se3_log(_compose(oracle.se3_exp(xi - e), Ti))
        fd[:, i] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(J, fd, atol=2e-8)


def test_left_jacobian_identity_at_zero():
    np.testing.assert_array_equal(oracle.se3_left_jacobian(np.zeros(6)), np.eye(6))


def test_pose_update_gradient_map_fd():
    """g_xi = Jl(xi)^T g_tangent equals the FD of L(Exp(xi) T0) for a linear
    L(T) = <tangent, Log-free first order perturbation>: we use the track
    loss as L."""
    rng = np.random.default_rng(3)
    cam0 = _cam(rng)
    T0 = np.concatenate([np.array(cam0.R[:]), np.array(cam0.t[:])])
    xi = rng.normal(0, 0.05, 6)
    X = rng.uniform(-1, 1, (20, 3))
    xy = rng.uniform(200, 400, (20, 2))

    def cam_of(x):
        T = _compose(oracle.se3_exp(x), T0)
        return oracle.make_camera(640, 480, cam0.fx, cam0.fy, cam0.cx, cam0.cy, T[:9], T[9:])

    def L(x):
        return oracle.track(X, np.arange(20), np.zeros(20), xy, [cam_of(x)])[0]

    _, _, tan, _ = oracle.track(X, np.arange(20), np.zeros(20), xy, [cam_of(xi)])
    g_xi, Rt = oracle.pose_update(T0[None], xi.copy(), tan, use_adam=False)
    h = 1e-6
    fd = np.array([(L(xi + h * e) - L(xi - h * e)) / (2 * h) for e in np.eye(6)])
    np.testing.assert_allclose(g_xi[0], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
    np.testing.assert_allclose(Rt[0], _compose(oracle.se3_exp(xi), T0), atol=1e-15)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    p = rng.normal(size=50)
    m, v = np.zeros(50), np.zeros(50)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 6):
        g = rng.normal(size=50)
        oracle.adam(p, g, m, v, 1e-3, 0.9, 0.999, 1e-15, step)
        tp.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-15)


def _sphere_quadrature(n_theta=24, n_phi=48):
    x, w = np.polynomial.legendre.leggauss(n_theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None]).reshape(-1)
    return dirs, wts


def test_sh_basis_orthonormal_and_harmonic_degree():
    """Gauss-Legendre x uniform quadrature (exact for these degrees):
    integral Y_a Y_b dOmega = delta_ab for all 16 functions; band l is a
    homogeneous polynomial of degree l (checked by scaling)."""
    dirs, wts = _sphere_quadrature()
    Y = np.stack([oracle.sh_eval(3, d)[0] for d in dirs])
    G = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)
    band = [0] + [1] * 3 + [2] * 5 + [3] * 7
    d = np.array([0.3, -0.5, 0.7])
    Y1 = oracle.sh_eval(3, d)[0]
    Y2 = oracle.sh_eval(3, 2.0 * d)[0]
    np.testing.assert_allclose(Y2, Y1 * 2.0 ** np.array(band), rtol=1e-12)


def test_sh_gradient_fd_and_degree0_view_independence():
    rng = np.random.default_rng(5)
    d = rng.normal(size=3)
    Y, dY = oracle.sh_eval(3, d)
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (oracle.sh_eval(3, d + e)[0] - oracle.sh_eval(3, d - e)[0]) / (2 * h)
        np.testing.assert_allclose(dY[:, i], fd, atol=1e-8)
    # degree 0: the colour does not depend on the camera position
    sc = oracle.Scene([[0.1, 0.0, 4.0]], [[-2.5] * 3], [[1, 0, 0, 0]], [0.5], [[[0.3, -0.2, 0.1]]])
    c1 = oracle.make_camera(64, 48, 60, 60, 32, 24, np.eye(3), [0, 0, 0])
    c2 = oracle.make_camera(64, 48, 60, 60, 32, 24, np.eye(3), [0.3, -0.2, 0.5])
    p1, p2 = oracle.project(sc, c1)[0], oracle.project(sc, c2)[0]
    assert p1[oracle.P["r"]] == p2[oracle.P["r"]] and p1[oracle.P["b"]] == p2[oracle.P["b"]]


def test_paper_constants_golden():
    """Hyperparameters the paper prints (tests/golden/paper_constants.json,
    each with its citation) are the defaults of the oracle-side helpers."""
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        gold = json.load(f)
    assert gold["huber_delta_px"]["value"] == 1.0
    loss_default, *_ = oracle.track([[0, 0, 2.0]], [0], [0], [[52.0, 50.0]],
                                    [oracle.make_camera(100, 100, 50, 50, 50, 50, np.eye(3), [0, 0, 0])])
    # default delta = 1 px: residual 2 px is in the linear branch (2*2-1)
    assert loss_default == pytest.approx(3.0)
    for key in ("lambda_ssim", "lambda_ba", "pose_lr", "t_max", "max_gaussians"):
        assert "cite" in gold[key] and gold[key]["value"] > 0
