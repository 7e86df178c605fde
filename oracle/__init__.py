"""FP64 CPU oracle for the joint 3DGS + pose + feature-track training step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2603_04847_gb300``) and imports
nothing from it.

The arithmetic lives in ``gs_oracle.c`` (plain C, double precision), built
here with gcc into ``liboracle.so`` and loaded through ctypes.  This module
only marshals numpy arrays and adds the discrete tile stage, which is a
plain lexicographic sort (a library primitive) over the oracle's own
projected records.

Passages restated (GloSplat, arXiv 2603.04847):
  * Eq. 5 (the photometric loss: its L1 part, and its SSIM part in numpy
    below) and Algorithm 1 "Rasterize";
  * Eq. 6 (Huber reprojection loss on track points, delta = 1 px);
  * the projection pi(K, T, X) = proj(K (R X + t)) after Algorithm 1;
  * T_i = T_i^(0) (+) dT_i (Algorithm 1), read as Exp(xi) T0;
  * one whole iteration of Algorithm 1 (joint_step): the pieces above
    composed in the algorithm's order, with Adam on every group.
  * Eq. 4 (the SfM bundle adjustment: Levenberg-Marquardt over SE(3) poses
    and points on the Huber reprojection objective), in ``ba.py``.
  * the MCMC densification rules the paper cites (Sec. 3.3), in ``mcmc.py``.
Where the paper leaves a point open the oracle takes the published 3DGS
convention its rasterizer follows, stated beside the code that applies it.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, library special cases and central finite
differences).  The paper's own quality numbers (PSNR etc.) need its datasets
and are not reproduced ("parity unpinned" for those only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4
RECT_MARGIN = 1.0 / 64.0   # px around a splat's support box (gs_oracle.c RECT_MARGIN)

PROJ_FIELDS = [
    "visible", "depth", "mx", "my", "cov_xx", "cov_xy", "cov_yy",
    "con_a", "con_b", "con_c", "opacity", "r", "g", "b",
    "bound_x0", "bound_y0", "bound_x1", "bound_y1",
    "px_x0", "px_y0", "px_x1", "px_y1", "xc", "yc",
]
P = {name: i for i, name in enumerate(PROJ_FIELDS)}

KNIFE_ALPHA_MIN = 1
KNIFE_T_MIN = 2
KNIFE_ALPHA_MAX = 4
KNIFE_DEPTH = 8


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into liboracle.so with gcc (portable flags only)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd, cwd=_HERE)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


class Camera(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double),
        ("cx", ctypes.c_double), ("cy", ctypes.c_double),
        ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
        ("near_plane", ctypes.c_double), ("far_plane", ctypes.c_double),
    ]


class _Scene(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
        ("mean", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
        ("quat", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p),
        ("sh", ctypes.c_void_p),
    ]


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.orc_sh_eval.argtypes = [ctypes.c_int, vp, vp, vp]
        lib.orc_project.argtypes = [vp, vp, vp]
        lib.orc_render.argtypes = [vp, vp, vp, i64, vp, dbl, vp, vp, vp, vp, vp, vp]
        lib.orc_render_tiled.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp]
        lib.orc_render_bwd.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.orc_track.argtypes = [i32, vp, i64, vp, vp, vp, i32, vp, dbl, dbl, vp, vp, vp, vp, vp]
        lib.orc_se3_exp.argtypes = [vp, vp]
        lib.orc_se3_log.argtypes = [vp, vp]
        lib.orc_se3_left_jacobian.argtypes = [vp, vp]
        lib.orc_adam.argtypes = [i64, vp, vp, vp, vp, dbl, dbl, dbl, dbl, ctypes.c_int]
        lib.orc_pose_update.argtypes = [i32, vp, vp, vp, vp, vp, vp, ctypes.c_int,
                                        dbl, dbl, dbl, dbl, ctypes.c_int, vp]
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data


def make_camera(width, height, fx, fy, cx, cy, R, t, near=0.01, far=1e10) -> Camera:
    c = Camera()
    c.width, c.height = int(width), int(height)
    c.fx, c.fy, c.cx, c.cy = float(fx), float(fy), float(cx), float(cy)
    R = np.asarray(R, dtype=np.float64).reshape(9)
    t = np.asarray(t, dtype=np.float64).reshape(3)
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    c.near_plane, c.far_plane = float(near), float(far)
    return c


def camera_from_rt(width, height, K, Rt, near=0.01, far=1e10) -> Camera:
    """K = (fx, fy, cx, cy); Rt = 12 numbers, row-major R then t."""
    Rt = np.asarray(Rt, dtype=np.float64).reshape(12)
    return make_camera(width, height, K[0], K[1], K[2], K[3], Rt[:9], Rt[9:], near, far)


class Scene:
    """Raw Gaussian parameters in double precision (keeps the arrays alive)."""

    def __init__(self, mean, log_scale, quat, opacity_logit, sh):
        self.mean = _f64(mean).reshape(-1, 3)
        self.log_scale = _f64(log_scale).reshape(-1, 3)
        self.quat = _f64(quat).reshape(-1, 4)
        self.opacity_logit = _f64(opacity_logit).reshape(-1)
        sh = _f64(sh)
        n = self.mean.shape[0]
        self.sh = sh.reshape(n, -1, 3)
        K = self.sh.shape[1]
        deg = int(round(np.sqrt(K))) - 1
        if (deg + 1) ** 2 != K or deg > 3:
            raise ValueError("sh must have (deg+1)^2 <= 16 coefficients per channel")
        self.sh_degree = deg
        self.n = n
        self._c = _Scene(n, deg, _ptr(self.mean), _ptr(self.log_scale), _ptr(self.quat),
                         _ptr(self.opacity_logit), _ptr(self.sh))

    @property
    def c(self):
        return ctypes.byref(self._c)

    def copy(self):
        return Scene(self.mean.copy(), self.log_scale.copy(), self.quat.copy(),
                     self.opacity_logit.copy(), self.sh.copy())


def sh_eval(degree, d):
    K = (degree + 1) ** 2
    Y = np.zeros(K)
    dY = np.zeros((K, 3))
    r = _L().orc_sh_eval(int(degree), _ptr(_f64(d)), _ptr(Y), _ptr(dY))
    if r < 0:
        raise ValueError("bad degree")
    return Y, dY


def project(scene: Scene, cam: Camera) -> np.ndarray:
    out = np.zeros((scene.n, len(PROJ_FIELDS)))
    _L().orc_project(scene.c, ctypes.byref(cam), _ptr(out))
    return out


def render(scene: Scene, cam: Camera, bg=(0.0, 0.0, 0.0), pixels=None, knife_eps=0.0):
    """Brute-force render of one view.  Returns dict with image [H,W,3] (or
    [npix,3]), T_final, last_id, n_added, knife flags and the pair count."""
    bg = _f64(bg)
    if pixels is None:
        npix = cam.width * cam.height
        pix = None
        shape = (cam.height, cam.width)
    else:
        pix = _i32(pixels).reshape(-1, 2)
        npix = pix.shape[0]
        shape = (npix,)
    image = np.zeros(shape + (3,))
    T = np.zeros(shape)
    last = np.zeros(shape, dtype=np.int32)
    nadd = np.zeros(shape, dtype=np.int32)
    knife = np.zeros(shape, dtype=np.int32)
    pairs = ctypes.c_int64(0)
    _L().orc_render(scene.c, ctypes.byref(cam), _ptr(bg), npix, _ptr(pix), float(knife_eps),
                    _ptr(image), _ptr(T), _ptr(last), _ptr(nadd), _ptr(knife),
                    ctypes.byref(pairs))
    return dict(image=image, T_final=T, last_id=last, n_added=nadd, knife=knife,
                n_pairs=pairs.value)


def render_tiled(scene: Scene, cam: Camera, tile: int, bg=(0.0, 0.0, 0.0)):
    bg = _f64(bg)
    image = np.zeros((cam.height, cam.width, 3))
    T = np.zeros((cam.height, cam.width))
    r = _L().orc_render_tiled(scene.c, ctypes.byref(cam), _ptr(bg), int(tile), _ptr(image), _ptr(T))
    if r != 0:
        raise ValueError("bad tile")
    return image, T


def render_bwd(scene: Scene, cam: Camera, v_image, bg=(0.0, 0.0, 0.0), pixels=None):
    """Gradients of sum(v_image * image) w.r.t. all raw parameters and the
    camera's left-perturbation pose tangent (6); tangent_abs is the sum of
    the absolute per-Gaussian tangent contributions."""
    bg = _f64(bg)
    v = _f64(v_image)
    if pixels is None:
        npix, pix = cam.width * cam.height, None
    else:
        pix = _i32(pixels).reshape(-1, 2)
        npix = pix.shape[0]
    v = v.reshape(npix, 3)
    n, K = scene.n, scene.sh.shape[1]
    g = dict(mean=np.zeros((n, 3)), log_scale=np.zeros((n, 3)), quat=np.zeros((n, 4)),
             opacity_logit=np.zeros(n), sh=np.zeros((n, K, 3)), tangent=np.zeros(6),
             tangent_abs=np.zeros(6), v2d=np.zeros((n, 9)))
    _L().orc_render_bwd(scene.c, ctypes.byref(cam), _ptr(bg), npix, _ptr(pix), _ptr(v),
                        _ptr(g["mean"]), _ptr(g["log_scale"]), _ptr(g["quat"]),
                        _ptr(g["opacity_logit"]), _ptr(g["sh"]), _ptr(g["tangent"]),
                        _ptr(g["tangent_abs"]), _ptr(g["v2d"]))
    return g


def l1_loss_grad(image, target, weight=1.0):
    """L1 part of Eq. 5 for one view: weight * mean |image - target| over
    pixels and channels, and its (sub)gradient with sign(0) = 0."""
    image = _f64(image)
    target = _f64(target)
    n = image.size
    d = image - target
    return weight * np.abs(d).sum() / n, weight * np.sign(d) / n


# SSIM of Eq. 5.  The paper names the term and its weight (lambda_SSIM = 0.2)
# but not the window; the oracle takes the structural similarity index of
# Wang et al. (2004) as 3DGS trains with it: an 11x11 Gaussian window with
# sigma = 1.5 (1-D taps normalised to sum 1), C1 = 0.01^2, C2 = 0.03^2
# (dynamic range 1), each colour channel on its own, zero padding outside the
# image with the window not renormalised there, and the mean of the SSIM map
# over pixels and channels.
SSIM_RADIUS = 5
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def ssim_window():
    """The 1-D taps w[-5..5] of the separable SSIM window."""
    k = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * SSIM_SIGMA * SSIM_SIGMA))
    return w / w.sum()


def window_sum(a):
    """sum over i, j in [-5, 5] of w[i] w[j] a[y + i, x + j] for every pixel
    (y, x) of a [H, W, C] array, with a = 0 outside the image."""
    a = _f64(a)
    H, W = a.shape[:2]
    r = SSIM_RADIUS
    w = ssim_window()
    pad = np.zeros((H + 2 * r, W + 2 * r) + a.shape[2:])
    pad[r:r + H, r:r + W] = a
    out = np.zeros_like(a)
    for i in range(2 * r + 1):
        for j in range(2 * r + 1):
            out += w[i] * w[j] * pad[i:i + H, j:j + W]
    return out


def ssim_map(x, y):
    """Per-pixel, per-channel SSIM of images x, y [H, W, C] and the local
    statistics it is made of (window means, variances, covariance)."""
    x, y = _f64(x), _f64(y)
    mx, my = window_sum(x), window_sum(y)
    vx = window_sum(x * x) - mx * mx
    vy = window_sum(y * y) - my * my
    cxy = window_sum(x * y) - mx * my
    A1 = 2.0 * mx * my + SSIM_C1
    A2 = 2.0 * cxy + SSIM_C2
    B1 = mx * mx + my * my + SSIM_C1
    B2 = vx + vy + SSIM_C2
    return A1 * A2 / (B1 * B2), dict(mx=mx, my=my, vx=vx, vy=vy, cxy=cxy, A1=A1, A2=A2, B1=B1, B2=B2)


def photo_loss_grad(image, target, l1_weight=0.8, ssim_weight=0.2):
    """Eq. 5 for one view (image, target [H, W, 3]):
        L = l1_weight * mean |x - y| + ssim_weight * (1 - mean SSIM(x, y))
    (lambda_SSIM = 0.2 gives the paper's weights 0.8 and 0.2) and dL/dx.

    The SSIM gradient is the chain rule through the window sums: with
    S = A1 A2 / (B1 B2) a function of the window means mx, my and of the
    window sums Exx = window_sum(x^2), Exy = window_sum(x y) (vx = Exx - mx^2,
    cxy = Exy - mx my), and g = -ssim_weight / n for n = H W C,
        M1 = g dS/dmx,  M2 = g dS/dExx,  M3 = g dS/dExy   (per pixel),
        dL/dx = window_sum(M1) + 2 x window_sum(M2) + y window_sum(M3),
    the window sum being its own adjoint (symmetric window, zero padding).
    The L1 part uses sign(0) = 0."""
    x, y = _f64(image), _f64(target)
    n = x.size
    S, st = ssim_map(x, y)
    mx, my, A1, A2, B1, B2 = st["mx"], st["my"], st["A1"], st["A2"], st["B1"], st["B2"]
    dS_dmx = 2.0 * my * A2 / (B1 * B2) - 2.0 * mx * S / B1   # vx, cxy held fixed
    dS_dvx = -S / B2
    dS_dcxy = 2.0 * A1 / (B1 * B2)
    g = -ssim_weight / n
    M1 = g * (dS_dmx - 2.0 * mx * dS_dvx - my * dS_dcxy)
    M2 = g * dS_dvx
    M3 = g * dS_dcxy
    grad = window_sum(M1) + 2.0 * x * window_sum(M2) + y * window_sum(M3)
    d = x - y
    grad = grad + l1_weight * np.sign(d) / n
    loss = l1_weight * np.abs(d).sum() / n + ssim_weight * (1.0 - S.sum() / n)
    return loss, grad


def track(X, obs_point, obs_cam, obs_xy, cams, delta=1.0, weight=1.0, with_abs=False):
    """Eq. 6 over the given observations.  Returns (sum rho, grad_X of
    weight*sum rho, pose tangents [n_cams,6], n_masked) and, with_abs, the
    per-camera sums of absolute tangent contributions."""
    X = _f64(X).reshape(-1, 3)
    op, oc = _i32(obs_point), _i32(obs_cam)
    xy = _f64(obs_xy).reshape(-1, 2)
    arr = (Camera * len(cams))(*cams)
    loss = ctypes.c_double(0.0)
    masked = ctypes.c_int64(0)
    gX = np.zeros_like(X)
    tan = np.zeros((len(cams), 6))
    tabs = np.zeros((len(cams), 6))
    r = _L().orc_track(X.shape[0], _ptr(X), op.shape[0], _ptr(op), _ptr(oc), _ptr(xy),
                       len(cams), arr, float(delta), float(weight), ctypes.byref(loss),
                       _ptr(gX), _ptr(tan), _ptr(tabs), ctypes.byref(masked))
    if r != 0:
        raise ValueError("observation index out of range")
    if with_abs:
        return loss.value, gX, tan, masked.value, tabs
    return loss.value, gX, tan, masked.value


def project_points(X, cam: Camera):
    """pi(K, T, X) for points X [n,3] (the projection after Algorithm 1);
    returns uv [n,2] and camera depth [n].  Used to synthesise noiseless
    track observations in tests."""
    X = _f64(X).reshape(-1, 3)
    R = np.array(cam.R[:]).reshape(3, 3)
    t = np.array(cam.t[:])
    Xc = X @ R.T + t
    uv = np.stack([cam.fx * Xc[:, 0] / Xc[:, 2] + cam.cx,
                   cam.fy * Xc[:, 1] / Xc[:, 2] + cam.cy], axis=1)
    return uv, Xc[:, 2]


def se3_exp(xi):
    T = np.zeros(12)
    _L().orc_se3_exp(_ptr(_f64(xi)), _ptr(T))
    return T


def se3_log(T):
    xi = np.zeros(6)
    _L().orc_se3_log(_ptr(_f64(T)), _ptr(xi))
    return xi


def se3_left_jacobian(xi):
    J = np.zeros(36)
    _L().orc_se3_left_jacobian(_ptr(_f64(xi)), _ptr(J))
    return J.reshape(6, 6)


def adam(p, g, m, v, lr, beta1=0.9, beta2=0.999, eps=1e-15, step=1):
    """In-place Adam step on float64 arrays p, m, v."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    _L().orc_adam(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), float(lr), float(beta1),
                  float(beta2), float(eps), int(step))


def pose_update(T0, xi, g_tangent, m=None, v=None, lr=1e-5, beta1=0.9, beta2=0.999,
                eps=1e-15, step=1, use_adam=True):
    """Returns (g_xi, Rt_out); xi, m, v are updated in place when use_adam."""
    T0 = _f64(T0).reshape(-1, 12)
    V = T0.shape[0]
    for a in (xi,) + ((m, v) if use_adam else ()):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gt = _f64(g_tangent).reshape(V, 6)
    g_xi = np.zeros((V, 6))
    Rt = np.zeros((V, 12))
    if m is None:
        m = np.zeros((V, 6))
    if v is None:
        v = np.zeros((V, 6))
    _L().orc_pose_update(V, _ptr(T0), _ptr(xi), _ptr(gt), _ptr(g_xi), _ptr(m), _ptr(v),
                         int(bool(use_adam)), float(lr), float(beta1), float(beta2),
                         float(eps), int(step), _ptr(Rt))
    return g_xi, Rt


def joint_step(params, X, T0, xi, wh, K, views, targets, obs_point, obs_view, obs_xy, hyper, state, step,
               merged_tracks=False, bg=(0.0, 0.0, 0.0)):
    """One iteration of Algorithm 1 (the joint optimisation loop) on a batch
    of views, in its order:
      1. compose the poses T_i = Exp(xi_i) T0_i                ("Apply pose adjustment");
      2. render every view of the batch and take the L1 part of Eq. 5,
         l1_weight * mean |I^ - I| per view, summed over the batch  ("Rasterize", "L_photo");
      3. the track term of Eq. 6 over the batch's observations, Huber with
         delta = huber_delta, weighted by lambda_BA (skipped at 0)  ("Joint BA loss");
      4. backpropagate both into the Gaussians, the track points and the
         per-camera pose tangents                                  ("Backpropagate");
      5. one Adam step on every Gaussian parameter group, on the track points
         and, unless freeze_poses, on the pose deltas (then recompose T_i)  ("Update").
    params: dict of the five raw Gaussian arrays (float64, updated copies are
    returned); X [K,3] track points (with merged_tracks the observations index
    the Gaussians and the track gradient goes into the means); T0 [V,12],
    xi [V,6]; targets: {view: image [H,W,3]}; obs_view holds each
    observation's camera; hyper: dict with lr_mean, lr_log_scale, lr_quat,
    lr_opacity, lr_sh, lr_track, lr_pose, beta1, beta2, eps, scene_extent,
    lambda_ba, huber_delta, l1_weight, freeze_poses; state: dict of Adam
    moments (created on first use, updated in place); step: the 1-based
    Adam step.  Returns dict(params, X, xi, Rt, grads, g_X, tangent,
    tangent_abs, loss_photo, loss_ba): the updated parameters, the
    gradients of the iteration (tangent_abs: the sums of the absolute
    per-term pose-tangent contributions) and the two loss terms (loss_ba the
    unweighted sum of rho)."""
    h = hyper
    p = {k: np.array(v, np.float64, copy=True) for k, v in params.items()}
    X = np.array(X, np.float64, copy=True)
    xi = np.array(xi, np.float64, copy=True).reshape(-1, 6)
    T0 = np.asarray(T0, np.float64).reshape(-1, 12)
    V = T0.shape[0]
    # 1. poses of this iteration
    Rt = np.stack([pose_update(T0[i:i + 1], xi[i:i + 1].copy(), np.zeros((1, 6)), use_adam=False)[1][0]
                   for i in range(V)])
    cams = [camera_from_rt(int(wh[i][0]), int(wh[i][1]), K[i], Rt[i]) for i in range(V)]
    sc = Scene(p["mean"], p["log_scale"], p["quat"], p["opacity_logit"], p["sh"])
    grads = {k: np.zeros_like(v) for k, v in p.items()}
    tangent = np.zeros((V, 6))
    tangent_abs = np.zeros((V, 6))
    loss_photo = 0.0
    # 2.-4. photometric term of every view of the batch and its backward
    for v in views:
        img = render(sc, cams[v], bg=bg)["image"]
        lv, dv = l1_loss_grad(img, targets[v], weight=h["l1_weight"])
        loss_photo += lv
        g = render_bwd(sc, cams[v], dv, bg=bg)
        for k in grads:
            grads[k] += g[k].reshape(grads[k].shape)
        tangent[v] += g["tangent"]
        tangent_abs[v] += g["tangent_abs"]
    # 3.-4. the track term over the observations of the batch's views
    loss_ba = 0.0
    g_X = np.zeros_like(p["mean"] if merged_tracks else X)
    if h["lambda_ba"] != 0.0:
        sel = np.isin(np.asarray(obs_view), np.asarray(views))
        pts = p["mean"] if merged_tracks else X
        loss_ba, g_X, tan_t, _, tabs = track(pts, np.asarray(obs_point)[sel], np.asarray(obs_view)[sel],
                                             np.asarray(obs_xy)[sel], cams, h["huber_delta"], h["lambda_ba"],
                                             with_abs=True)
        tangent += tan_t
        tangent_abs += tabs
        if merged_tracks:
            grads["mean"] += g_X
    # 5. Adam on every group, then the poses
    ext = h["scene_extent"]
    lrs = dict(mean=h["lr_mean"] * ext, log_scale=h["lr_log_scale"], quat=h["lr_quat"],
               opacity_logit=h["lr_opacity"], sh=h["lr_sh"])
    for k in p:
        m = state.setdefault("m_" + k, np.zeros(p[k].size))
        vv = state.setdefault("v_" + k, np.zeros(p[k].size))
        flat = p[k].reshape(-1).copy()
        adam(flat, grads[k].reshape(-1), m, vv, lrs[k], h["beta1"], h["beta2"], h["eps"], step)
        p[k] = flat.reshape(p[k].shape)
    if not merged_tracks:
        m = state.setdefault("m_X", np.zeros(X.size))
        vv = state.setdefault("v_X", np.zeros(X.size))
        flat = X.reshape(-1).copy()
        adam(flat, g_X.reshape(-1), m, vv, h["lr_track"] * ext, h["beta1"], h["beta2"], h["eps"], step)
        X = flat.reshape(X.shape)
    else:
        X = p["mean"]
    Rt_new = Rt
    if not h["freeze_poses"]:
        m = state.setdefault("m_xi", np.zeros((V, 6)))
        vv = state.setdefault("v_xi", np.zeros((V, 6)))
        _, Rt_new = pose_update(T0, xi, tangent, m, vv, lr=h["lr_pose"], beta1=h["beta1"], beta2=h["beta2"],
                                eps=h["eps"], step=step)
    return dict(params=p, X=X, xi=xi, Rt=Rt_new, grads=grads, g_X=g_X, tangent=tangent, tangent_abs=tangent_abs,
                loss_photo=loss_photo, loss_ba=loss_ba)


def tile_lists(proj: np.ndarray, width: int, height: int, tile: int):
    """Discrete stage: every (tile, depth, index) instance of one view from
    the oracle's own pixel rectangles, in the canonical order (tile, depth
    ascending, index ascending).  Returns (tile_id, depth, gid) arrays."""
    vis = proj[:, P["visible"]] > 0
    idx = np.nonzero(vis)[0]
    tiles_x = (width + tile - 1) // tile
    tl, dl, gl = [], [], []
    for j in idx:
        x0 = int(proj[j, P["px_x0"]]) // tile
        y0 = int(proj[j, P["px_y0"]]) // tile
        x1 = int(proj[j, P["px_x1"]]) // tile
        y1 = int(proj[j, P["px_y1"]]) // tile
        for ty in range(y0, y1 + 1):
            for tx in range(x0, x1 + 1):
                tl.append(ty * tiles_x + tx)
                dl.append(proj[j, P["depth"]])
                gl.append(j)
    t = np.array(tl, dtype=np.int64)
    d = np.array(dl, dtype=np.float64)
    g = np.array(gl, dtype=np.int64)
    order = np.lexsort((g, d, t))
    return t[order], d[order], g[order]
