"""The torch.autograd.Function wrappers: gradcheck against finite
differences on a tiny knife-edge-free scene (FP32 kernels, float64 finite
differences, FP32-appropriate tolerances), and autograd gradients —
including d/dxi of the pose deltas — against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import f32, knife_mask, oracle_cam, oracle_scene, pose_rel_err, rel_linf
from test_oracle_grad import smooth_camera, smooth_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _cams_from_oracle(cam):
    from paper_2603_04847_gb300 import Cameras
    Rt = np.concatenate([np.array(cam.R[:]), np.array(cam.t[:])])[None]
    return Cameras.from_numpy([[cam.width, cam.height]], [[cam.fx, cam.fy, cam.cx, cam.cy]], Rt), Rt


def test_render_gradcheck_tiny_smooth_scene():
    from paper_2603_04847_gb300.autograd import RenderState, render
    rng = np.random.default_rng(0)
    sc = smooth_scene(rng, n=5, sh_degree=2)
    cam = smooth_camera(rng)
    cams, Rt = _cams_from_oracle(cam)
    state = RenderState(cams, [0])
    dev = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda", requires_grad=True)
    params = [dev(sc.mean), dev(sc.log_scale), dev(sc.quat), dev(sc.opacity_logit), dev(sc.sh),
              dev(rng.normal(0, 0.01, (1, 6)))]
    T0 = torch.tensor(Rt, dtype=torch.float32, device="cuda")
    w = torch.tensor(rng.normal(size=(20 * 24, 3)), dtype=torch.float64, device="cuda")

    def f(*p):
        return (render(*p, T0, state) * w).sum()

    assert torch.autograd.gradcheck(f, params, eps=1e-3, atol=5e-3, rtol=2e-2, nondet_tol=1e-5)


def test_render_autograd_matches_oracle():
    """Autograd of <w, render(params, xi)> on the 256x192 / 2k workload at a
    non-zero pose delta: parameter gradients against the oracle, and
    d/dxi against Jl(xi)^T of the oracle's pose tangent."""
    from paper_2603_04847_gb300 import Cameras
    from paper_2603_04847_gb300.autograd import RenderState, render
    w = synth.make_workload("tiny")
    sc, wh, K, Rt0 = w["scene"], w["wh"], w["K"], w["Rt"]
    xi = f32(np.array([[0.01, -0.02, 0.03, 0.004, -0.003, 0.002]]))
    Rt_xi = oracle.pose_update(f32(Rt0), xi.copy(), np.zeros((1, 6)), use_adam=False)[1]
    cam = oracle_cam(wh, K, Rt_xi, 0)
    osc = oracle_scene(sc)
    ref = oracle.render(osc, cam, knife_eps=1e-4)
    rng = np.random.default_rng(2)
    wv = f32(rng.normal(size=(192, 256, 3)))
    wv[knife_mask(ref)] = 0.0
    cams = Cameras.from_numpy(wh, K, Rt0)
    state = RenderState(cams, [0])
    dev = lambda a: torch.tensor(f32(a), dtype=torch.float32, device="cuda", requires_grad=True)
    params = [dev(sc[k]) for k in ("mean", "log_scale", "quat", "opacity_logit", "sh")]
    xit = dev(xi)
    img = render(*params, xit, cams.Rt, state)
    img.backward(torch.tensor(wv.reshape(-1, 3), dtype=torch.float32, device="cuda"))
    exp = oracle.render_bwd(osc, cam, wv)
    for p, name in zip(params, ("mean", "log_scale", "quat", "opacity_logit", "sh")):
        assert rel_linf(p.grad.cpu().numpy(), exp[name]) <= 1e-3, name
    g_xi_o, _ = oracle.pose_update(f32(Rt0), xi.copy(), exp["tangent"][None], use_adam=False)
    got = xit.grad.cpu().numpy()[0].astype(np.float64)
    # map the pose-tangent scale through Jl^T (near identity for this small xi)
    assert pose_rel_err(got, g_xi_o[0], exp["tangent_abs"]) <= 1e-3


def test_track_loss_autograd_matches_oracle():
    from paper_2603_04847_gb300 import Batch, Cameras
    from paper_2603_04847_gb300.autograd import track_loss
    w = synth.make_workload("train", n_gaussians=5000, n_views=6, n_tracks=500)
    wh, K, Rt0 = w["wh"], w["K"], w["Rt"]
    tr = w["tracks"]
    rng = np.random.default_rng(3)
    xi = f32(rng.normal(0, 0.01, (6, 6)))
    Rt_xi = oracle.pose_update(f32(Rt0), xi.copy(), np.zeros((6, 6)), use_adam=False)[1]
    cams_o = [oracle_cam(wh, K, Rt_xi, v) for v in range(6)]
    X = f32(tr["X"])
    xy = f32(rng.uniform(0, 1, (len(tr["obs_point"]), 2)) * wh[tr["obs_view"]])
    views = [1, 4, 5]
    sel = np.isin(tr["obs_view"], views)
    lo, gX, tan, _, tabs = oracle.track(X, tr["obs_point"][sel], tr["obs_view"][sel], xy[sel], cams_o, 1.0, 0.1,
                                        with_abs=True)
    g_xi_o, _ = oracle.pose_update(f32(Rt0), xi.copy(), tan, use_adam=False)
    cams = Cameras.from_numpy(wh, K, Rt0)
    batch = Batch(cams, views)
    dev = lambda a, dt=torch.float32, rg=False: torch.tensor(np.asarray(a), dtype=dt, device="cuda", requires_grad=rg)
    Xt, xit = dev(X, rg=True), dev(xi, rg=True)
    L = track_loss(Xt, xit, cams.Rt, dev(tr["obs_point"], torch.int32), dev(xy), dev(tr["view_obs_offset"], torch.int64),
                   cams, batch, 1.0, 0.1)
    L.backward()
    assert L.item() == pytest.approx(0.1 * lo, rel=1e-5)
    assert rel_linf(Xt.grad.cpu().numpy(), gX) <= 1e-3
    for v in views:
        assert pose_rel_err(xit.grad.cpu().numpy()[v].astype(np.float64), g_xi_o[v], tabs[v]) <= 1e-3
