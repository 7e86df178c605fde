"""Pins of the oracle's forward renderer against closed forms, invariants and
brute force (no GPU).  The oracle restates the rasterizer that Sec. 3.3 of
the paper delegates to gsplat, with that rasterizer's published conventions
where the paper is silent."""
import math

import numpy as np
import pytest

import oracle
import synth


def _identity_cam(W=256, H=192, f=220.0):
    return oracle.make_camera(W, H, f, f, W / 2.0, H / 2.0, np.eye(3), [0, 0, 0])


def _random_unit_quat(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q) * rng.uniform(0.5, 2.0)  # unnormalised on purpose


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_isotropic_splat_closed_form(seed):
    """One isotropic Gaussian at (0,0,z0), identity camera, f=220: the 2-D
    covariance is ((f s / z0)^2 + 0.3) I, the mean projects to the principal
    point and every pixel is c * min(0.99, o exp(-r^2 / (2 sigma'^2))) where
    that is >= 1/255 (background 0), T_final = 1 - alpha."""
    rng = np.random.default_rng(seed)
    z0 = rng.uniform(3, 6)
    s = rng.uniform(0.02, 0.08)
    ologit = rng.normal()
    cam = _identity_cam()
    sc = oracle.Scene([[0, 0, z0]], [[math.log(s)] * 3], [_random_unit_quat(rng)], [ologit],
                      np.zeros((1, 1, 3)))  # SH zero -> colour 0.5 exactly
    r = oracle.render(sc, cam)
    sig2 = (220.0 * s / z0) ** 2 + 0.3
    o = 1.0 / (1.0 + math.exp(-ologit))
    v, u = np.mgrid[0:192, 0:256]
    r2 = (u + 0.5 - 128.0) ** 2 + (v + 0.5 - 96.0) ** 2
    a = np.minimum(0.99, o * np.exp(-0.5 * r2 / sig2))
    a = np.where(a >= 1.0 / 255.0, a, 0.0)
    np.testing.assert_allclose(r["image"][..., 0], 0.5 * a, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["image"][..., 2], 0.5 * a, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["T_final"], 1.0 - a, rtol=1e-12, atol=1e-15)
    p = oracle.project(sc, cam)[0]
    assert p[oracle.P["mx"]] == pytest.approx(128.0, abs=1e-12)
    assert p[oracle.P["my"]] == pytest.approx(96.0, abs=1e-12)
    np.testing.assert_allclose([p[oracle.P["cov_xx"]], p[oracle.P["cov_xy"]], p[oracle.P["cov_yy"]]],
                               [sig2, 0.0, sig2], rtol=1e-10, atol=1e-12)


def test_two_cocentred_splats_over_operator_and_depth_swap():
    """C = c1 a1 + c2 a2 (1 - a1) at the centre; swapping depths swaps order."""
    cam = _identity_cam()
    Y00 = 0.5 / math.sqrt(math.pi)  # textbook real SH Y_0^0
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    sh = np.stack([((c1 - 0.5) / Y00)[None], ((c2 - 0.5) / Y00)[None]])
    for za, zb in [(3.0, 5.0), (5.0, 3.0)]:
        sc = oracle.Scene([[0, 0, za], [0, 0, zb]], [[math.log(0.05)] * 3, [math.log(0.07)] * 3],
                          [[1, 0, 0, 0], [1, 0, 0, 0]], [0.3, -0.2], sh)
        # centre of pixel (127.5, 95.5) is offset by 0.5 px from the mean
        r = oracle.render(sc, cam, pixels=[[127, 95]])
        p = oracle.project(sc, cam)
        alphas = []
        for j in range(2):
            o = p[j, oracle.P["opacity"]]
            q = p[j, oracle.P["con_a"]] * 0.25 + 2 * p[j, oracle.P["con_b"]] * 0.25 + p[j, oracle.P["con_c"]] * 0.25
            alphas.append(min(0.99, o * math.exp(-0.5 * q)))
        front, back = (0, 1) if za < zb else (1, 0)
        cols = [c1, c2]
        want = cols[front] * alphas[front] + cols[back] * alphas[back] * (1 - alphas[front])
        np.testing.assert_allclose(r["image"][0], want, rtol=1e-12)
        assert r["last_id"][0] == back


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tiled_equals_untiled(tile):
    """The opacity-aware rectangle is conservative, so compositing per tile
    over the Gaussians whose rectangle meets it gives the untiled image bit
    for bit (support rule independent of the tile size)."""
    w = synth.make_workload("tiny", n_gaussians=600)
    sc = oracle.Scene(**w["scene"])
    cam = oracle.camera_from_rt(256, 192, w["K"][0], w["Rt"][0])
    ref = oracle.render(sc, cam)
    img, T = oracle.render_tiled(sc, cam, tile)
    assert np.array_equal(img, ref["image"])
    assert np.array_equal(T, ref["T_final"])


def test_rect_is_conservative_brute_force():
    """Brute force over every pixel: each pixel where a Gaussian's alpha is
    >= 1/255 lies inside its rectangle, and the rectangle exceeds the exact
    support's bounding box by at most the 1/64-px margin (+1 rounding)."""
    rng = np.random.default_rng(5)
    n = 40
    cam = oracle.make_camera(64, 48, 60, 60, 32, 24, np.eye(3), [0, 0, 0])
    mean = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.2, 1.2, n), rng.uniform(2, 5, n)], 1)
    sc = oracle.Scene(mean, rng.normal(-2.0, 0.5, (n, 3)), rng.normal(size=(n, 4)),
                      rng.normal(0, 1.5, n), np.zeros((n, 1, 3)))
    p = oracle.project(sc, cam)
    v, u = np.mgrid[0:48, 0:64]
    for j in range(n):
        one = oracle.Scene(mean[j:j + 1], sc.log_scale[j:j + 1], sc.quat[j:j + 1],
                           sc.opacity_logit[j:j + 1], np.zeros((1, 1, 3)))
        T = oracle.render(one, cam)["T_final"]
        covered = T < 1.0  # alpha >= 1/255 somewhere on that pixel
        if not p[j, oracle.P["visible"]]:
            assert not covered.any()
            continue
        x0, y0, x1, y1 = (int(p[j, oracle.P[k]]) for k in ("px_x0", "px_y0", "px_x1", "px_y1"))
        inside = (u >= x0) & (u <= x1) & (v >= y0) & (v <= y1)
        assert not (covered & ~inside).any()
        b = [p[j, oracle.P[k]] for k in ("bound_x0", "bound_y0", "bound_x1", "bound_y1")]
        unclipped = b[0] > 1 and b[1] > 1 and b[2] < 62 and b[3] < 46
        if covered.any() and unclipped:
            uu, vv = u[covered], v[covered]
            assert uu.min() - x0 <= 2 and x1 - uu.max() <= 2
            assert vv.min() - y0 <= 2 and y1 - vv.max() <= 2


def test_transmittance_bounds():
    """T_final in [1e-4, 1]: the stop comes before T' < 1e-4.  (T_final is
    not monotone under adding an occluder, because of that stop.)"""
    w = synth.make_workload("tiny", n_gaussians=2000)
    sc = oracle.Scene(**w["scene"])
    cam = oracle.camera_from_rt(256, 192, w["K"][0], w["Rt"][0])
    r = oracle.render(sc, cam)
    assert r["T_final"].min() >= 1e-4 and r["T_final"].max() <= 1.0
    assert (r["n_added"] > 0).mean() > 0.3


def test_near_far_and_off_screen_cull():
    cam = _identity_cam()
    sc = oracle.Scene([[0, 0, 0.005], [0, 0, -2], [100, 0, 4], [0, 0, 4]], [[-3.0] * 3] * 4,
                      [[1, 0, 0, 0]] * 4, [0.0] * 4, np.zeros((4, 1, 3)))
    p = oracle.project(sc, cam)
    assert list(p[:, oracle.P["visible"]]) == [0, 0, 0, 1]
    # opacity below 1/255 is culled
    sc2 = oracle.Scene([[0, 0, 4]], [[-3.0] * 3], [[1, 0, 0, 0]], [math.log((1 / 256) / (1 - 1 / 256))],
                       np.zeros((1, 1, 3)))
    assert oracle.project(sc2, cam)[0, oracle.P["visible"]] == 0


def test_tile_lists_canonical_order():
    """Discrete stage: instances sorted by (tile, depth, index); the per-tile
    lists equal a brute-force enumeration of rectangles meeting each tile."""
    w = synth.make_workload("tiny", n_gaussians=300)
    sc = oracle.Scene(**w["scene"])
    cam = oracle.camera_from_rt(256, 192, w["K"][0], w["Rt"][0])
    p = oracle.project(sc, cam)
    t, d, g = oracle.tile_lists(p, 256, 192, 16)
    assert np.all(np.diff(t) >= 0)
    for tile_id in np.unique(t)[:50]:
        sel = t == tile_id
        ty, tx = divmod(int(tile_id), 16)
        brute = []
        for j in range(sc.n):
            if not p[j, oracle.P["visible"]]:
                continue
            x0, y0, x1, y1 = (int(p[j, oracle.P[k]]) for k in ("px_x0", "px_y0", "px_x1", "px_y1"))
            if x0 // 16 <= tx <= x1 // 16 and y0 // 16 <= ty <= y1 // 16:
                brute.append((p[j, oracle.P["depth"]], j))
        brute.sort()
        assert [j for _, j in brute] == list(g[sel])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_anisotropic_covariance_matches_scipy_rotation(seed):
    """A Gaussian on the optical axis of an identity camera: the 2-D
    covariance is (f/z)^2 [R diag(s^2) R^T]_{xy block} + 0.3 I, with R from
    scipy's quaternion-to-matrix (a library routine, scalar-last order)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    q = rng.normal(size=4)  # (w, x, y, z), unnormalised
    s = rng.uniform(0.02, 0.1, 3)
    z0 = 4.0
    cam = _identity_cam()
    sc = oracle.Scene([[0, 0, z0]], [np.log(s)], [q], [1.0], np.zeros((1, 1, 3)))
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    S = R @ np.diag(s ** 2) @ R.T
    want = (220.0 / z0) ** 2 * S[:2, :2] + 0.3 * np.eye(2)
    p = oracle.project(sc, cam)[0]
    got = np.array([[p[oracle.P["cov_xx"]], p[oracle.P["cov_xy"]]], [p[oracle.P["cov_xy"]], p[oracle.P["cov_yy"]]]])
    np.testing.assert_allclose(got, want, rtol=1e-12)
    inv = np.linalg.inv(want)
    np.testing.assert_allclose([p[oracle.P["con_a"]], p[oracle.P["con_b"]], p[oracle.P["con_c"]]],
                               [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-12)


def test_camera_world_equivariance():
    """Rendering with camera (R, t) equals rendering the scene moved into the
    camera frame (mu' = R mu + t, Gaussian rotation composed with R via
    scipy) with the identity camera (SH degree 0, so colour is
    view-independent)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(11)
    n = 50
    mean = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)], 1)
    q = rng.normal(size=(n, 4))
    ls = rng.normal(-2.5, 0.3, (n, 3))
    ol = rng.normal(0, 1, n)
    sh = rng.uniform(-1.5, 1.5, (n, 1, 3))
    Rc = Rotation.from_rotvec(rng.normal(0, 0.4, 3))
    t = np.array([0.1, -0.2, 4.0])
    cam = oracle.make_camera(96, 80, 90, 92, 47.5, 40.2, Rc.as_matrix(), t)
    ref = oracle.render(oracle.Scene(mean, ls, q, ol, sh), cam)["image"]
    mean2 = mean @ Rc.as_matrix().T + t
    rq = Rc * Rotation.from_quat(q[:, [1, 2, 3, 0]])
    q2 = rq.as_quat()[:, [3, 0, 1, 2]]
    cam0 = oracle.make_camera(96, 80, 90, 92, 47.5, 40.2, np.eye(3), [0, 0, 0])
    img = oracle.render(oracle.Scene(mean2, ls, q2, ol, sh), cam0)["image"]
    np.testing.assert_allclose(img, ref, atol=1e-9)
