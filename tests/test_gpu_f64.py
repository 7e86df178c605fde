"""The FP64 instantiation of the projection and compositing kernels (the
*_f64 entry points): the same kernels computing in double.

- Against the FP64 oracle they agree to double-precision rounding (images
  1e-12, gradients 1e-9 relative, pose tangent 1e-9 of its contribution
  scale), on the tiny scene and on the thin-streak scene whose FP32
  gradients lose digits to conditioning -- so the method as implemented is
  exact and the FP32 bars measure precision only.
- torch.autograd.gradcheck on 500 Gaussians with SH degree 3 and a pose
  delta, at gradcheck's default tolerances (eps 1e-6, atol 1e-5, rtol 1e-3):
  full mode over every geometric and opacity parameter and the pose, fast
  mode over all parameters including the SH coefficients.  The scene is
  built so that no finite-difference step crosses a discontinuity of the
  method (the alpha >= 1/255 cut, the T < 1e-4 stop, the 0.99 clamp, a
  change of depth order or of tile coverage): every splat covers the whole
  48x36 image with alpha between 0.0044 and 0.014 (the cut is 0.0039), the
  transmittance stays above 4e-3, no evaluated alpha or transmittance lies
  within 1e-3 (relative) of a threshold, and depths are at least 1.2e-3
  apart.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import f32, knife_mask, oracle_cam, oracle_scene, pose_rel_err, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("mean", "log_scale", "quat", "opacity_logit", "sh")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _f64_render(sc, wh, K, Rt, views, tile=16):
    from paper_2603_04847_gb300 import Batch, Cameras, Gaussians, Renderer
    g = Gaussians.from_numpy(sc, dtype=torch.float64)
    cams = Cameras.from_numpy(wh, K, Rt)
    Rt64 = torch.as_tensor(np.asarray(Rt, np.float64), device="cuda").contiguous()
    batch = Batch(cams, views, tile=tile)
    r = Renderer(g.n, cams, batch, dtype=torch.float64)
    r.ensure_capacity(g, Rt64)
    r.forward(g, Rt64)
    torch.cuda.synchronize()
    return r, g, Rt64


def _f64_backward(r, g, Rt64, v_image):
    from paper_2603_04847_gb300 import Gaussians
    dg = Gaussians.zeros_like(g)
    g_tan = torch.zeros((r.cams.V, 6), dtype=torch.float64, device="cuda")
    r.backward(g, dg, g_tan, v_image=torch.as_tensor(np.ascontiguousarray(v_image), device="cuda"), Rt=Rt64)
    torch.cuda.synchronize()
    out = {k: t.cpu().numpy() for k, t in zip(NAMES, dg.tensors())}
    out["tangent"] = g_tan.cpu().numpy()
    return out


@pytest.mark.parametrize("thin", [False, True])
@pytest.mark.parametrize("tile", [16, 32])
def test_f64_kernels_match_the_oracle_to_rounding(thin, tile):
    w = synth.make_workload("tiny")
    sc = {k: f32(v) for k, v in w["scene"].items()}
    if thin:   # every Gaussian a long thin streak (axes x e^2, e^-1.5, e^-1.5);
        # rounded to float like every input of the oracle (oracle_scene), so
        # that both sides see the same values
        sc["log_scale"] = f32(sc["log_scale"] + np.array([2.0, -1.5, -1.5]))
    wh, K, Rt = w["wh"], f32(w["K"]), f32(w["Rt"])
    r, g, Rt64 = _f64_render(sc, wh, K, Rt, [0], tile)
    cam = oracle_cam(wh, K, Rt, 0)
    osc = oracle_scene(sc)
    # knife edges at FP64 rounding, and depths within float rounding of
    # each other (the shared sort keys them on the float depth)
    ref = oracle.render(osc, cam, knife_eps=2e-7)
    ok = ~knife_mask(ref)
    assert (~ok).mean() < 2e-3
    img = r.image.cpu().numpy().reshape(192, 256, 3)
    assert rel_linf(img[ok], ref["image"][ok]) <= 1e-12
    np.testing.assert_allclose(r.T_final.cpu().numpy().reshape(192, 256)[ok], ref["T_final"][ok], rtol=1e-12)
    rng = np.random.default_rng(4)
    wv = rng.normal(size=(192, 256, 3))
    wv[~ok] = 0.0
    got = _f64_backward(r, g, Rt64, wv.reshape(-1, 3))
    exp = oracle.render_bwd(osc, cam, wv)
    for k in NAMES:
        assert rel_linf(got[k], exp[k]) <= 1e-9, (k, rel_linf(got[k], exp[k]))
    assert pose_rel_err(got["tangent"][0], exp["tangent"], exp["tangent_abs"]) <= 1e-9


def _smooth_500(rng, n=500, W=48, H=36):
    """500 broad, faint Gaussians in front of an identity camera (f = 45):
    2-D footprint sigma ~ 60 px, so alpha = o exp(-q/2) with q <= ~0.5 over
    the image; o ~ U(0.008, 0.014); depths on a jittered grid over [3, 6]."""
    k = np.arange(n)
    z = 3.0 + 3.0 * (k + rng.uniform(0.2, 0.8, n)) / n
    rng.shuffle(z)
    xy = rng.uniform(-0.08, 0.08, (n, 2)) * z[:, None]
    mean = np.concatenate([xy, z[:, None]], 1)
    log_scale = np.log(4.5) + rng.uniform(-0.15, 0.15, (n, 3))
    quat = rng.normal(size=(n, 4))
    o = rng.uniform(0.008, 0.014, n)
    opacity_logit = np.log(o / (1.0 - o))
    sh = np.zeros((n, 16, 3))
    sh[:, 0] = (rng.uniform(0.25, 0.75, (n, 3)) - 0.5) / 0.28209479177387814
    sh[:, 1:] = rng.normal(0.0, 0.02, (n, 15, 3))
    wh = np.array([[W, H]])
    K = np.array([[45.0, 45.0, W / 2.0, H / 2.0]])
    Rt = np.zeros((1, 12))
    Rt[0, [0, 4, 8]] = 1.0
    return dict(mean=mean, log_scale=log_scale, quat=quat, opacity_logit=opacity_logit, sh=sh), wh, K, Rt


def test_smooth_500_scene_is_free_of_discontinuities():
    """The gradcheck scene's margins, checked on the oracle: every pixel
    composites all 500 splats, no evaluated alpha or transmittance within
    1e-3 (relative) of 1/255, 0.99 or 1e-4 (no knife edge), T_final > 4e-3,
    opacities in [0.0075, 0.015], colours unclamped."""
    sc, wh, K, Rt = _smooth_500(np.random.default_rng(7))
    cam = oracle_cam(wh, K, Rt, 0)
    res = oracle.render(oracle.Scene(**sc), cam, knife_eps=1e-3)
    assert not res["knife"].any()
    assert (res["n_added"] == 500).all()
    assert res["T_final"].min() > 4e-3
    proj = oracle.project(oracle.Scene(**sc), cam)
    assert (proj[:, oracle.P["opacity"]] < 0.015).all() and (proj[:, oracle.P["opacity"]] > 0.0075).all()
    assert (proj[:, oracle.P["r"]] > 0.1).all()   # no colour clamp


def test_gradcheck_500_gaussians_fp64():
    from paper_2603_04847_gb300 import Cameras
    from paper_2603_04847_gb300.autograd import RenderState, render
    rng = np.random.default_rng(7)
    sc, wh, K, Rt = _smooth_500(rng)
    cams = Cameras.from_numpy(wh, K, Rt)
    state = RenderState(cams, [0], fixed_capacity=True)
    dev = lambda a, rg=True: torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda", requires_grad=rg)
    T0 = torch.tensor(Rt, dtype=torch.float64, device="cuda")
    wimg = torch.tensor(rng.normal(size=(48 * 36, 3)), dtype=torch.float64, device="cuda")
    xi = dev(rng.normal(0, 0.005, (1, 6)))
    geo = [dev(sc[k]) for k in ("mean", "log_scale", "quat", "opacity_logit")]
    sh = dev(sc["sh"])

    def f_geo(mean, log_scale, quat, opacity_logit, xi):
        return (render(mean, log_scale, quat, opacity_logit, sh.detach(), xi, T0, state) * wimg).sum()

    # full mode: every one of the 500 x 11 geometric / opacity parameters
    # and the 6 pose parameters, one by one
    assert torch.autograd.gradcheck(f_geo, geo + [xi], nondet_tol=1e-12)

    def f_all(mean, log_scale, quat, opacity_logit, sh, xi):
        return (render(mean, log_scale, quat, opacity_logit, sh, xi, T0, state) * wimg).sum()

    # fast mode over all 29,506 parameters including the SH coefficients
    assert torch.autograd.gradcheck(f_all, geo + [sh, xi], fast_mode=True, nondet_tol=1e-12)
