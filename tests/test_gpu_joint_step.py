"""One whole iteration of Algorithm 1 on the GPU -- JointStep captured in a
CUDA graph and replayed, the timed path: pose composition, projection,
sort, compositing, fused L1 and its backward, the track term on the side
stream, the pose update beside Adam on every parameter group -- against the
oracle's iteration (oracle.joint_step) on the same float32-rounded inputs,
for the full method and the paper's ablation variants (frozen poses,
photometric only, merged tracks), on the tiny workload and on a small batch
of uneven views laid out on the device.

Compared: both loss terms; every gradient of the iteration (Gaussians,
track points, per-camera pose tangents) at the usual bars; the parameters
after the Adam steps.  A first Adam step moves each parameter by about
-lr sign(g), so parameters are compared element by element where the
gradient is clearly non-zero (|g| >= 1e-2 max |g| of its tensor) and
within 2 lr elsewhere."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import f32, oracle_cam, pose_rel_err, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")
HYPER = dict(lr_mean=1.6e-4, lr_log_scale=5e-3, lr_quat=1e-3, lr_opacity=5e-2, lr_sh=2.5e-3, lr_track=1.6e-4,
             lr_pose=1e-4, beta1=0.9, beta2=0.999, eps=1e-15, scene_extent=1.0, lambda_ba=0.1, huber_delta=1.0,
             l1_weight=1.0, freeze_poses=False)
VARIANTS = {"full": {}, "frozen_poses": dict(freeze_poses=True), "photometric_only": dict(lambda_ba=0.0),
            "merged_tracks": {}}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _workload(kind):
    if kind == "tiny":
        w = synth.make_workload("tiny", n_gaussians=1500, n_tracks=150)
        return w, [0]
    w = synth.make_workload("batched", n_gaussians=3000, n_views=5, width=(80, 160), height=(64, 120),
                            n_tracks=200, seed=0)
    return w, [4, 1, 3]


def _inputs(w, merged):
    rng = np.random.default_rng(5)
    wh, K, Rt = w["wh"], f32(w["K"]), f32(w["Rt"])
    V = len(wh)
    params = {k: f32(v) for k, v in w["scene"].items()}
    gt = oracle.Scene(**{k: f32(v) for k, v in w["gt"].items()})
    targets = {v: f32(oracle.render(gt, oracle_cam(wh, K, Rt, v))["image"]) for v in range(V)}
    tr = w["tracks"]
    obs_point = tr["obs_point"].astype(np.int32)
    obs_view = tr["obs_view"].astype(np.int32)
    if merged:   # track k is Gaussian idx[k]: its point is that Gaussian's mean
        idx = rng.choice(len(params["mean"]), size=int(obs_point.max()) + 1, replace=False)
        obs_point = idx[obs_point].astype(np.int32)
        X = params["mean"]
    else:
        X = f32(tr["X"])
    xy = np.stack([oracle.project_points(X[k:k + 1], oracle_cam(wh, K, Rt, v))[0][0]
                   for k, v in zip(obs_point, obs_view)])
    xy = f32(xy + rng.normal(0, 1.5, xy.shape))    # residuals on both sides of delta = 1 px
    return params, X, wh, K, Rt, targets, obs_point, obs_view, xy, tr["view_obs_offset"]


def _gpu_step(w, views, inputs, hyper, merged, deterministic=False, replays=1):
    from paper_2603_04847_gb300 import Cameras, Gaussians, Hyper, JointStep
    params, X, wh, K, Rt, targets, obs_point, obs_view, xy, voff = inputs
    cams = Cameras.from_numpy(wh, K, Rt)
    g = Gaussians.from_numpy(params)
    P = (wh[:, 0] * wh[:, 1]).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(P)])
    tg = np.concatenate([targets[v].reshape(-1, 3) for v in range(len(wh))])
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    h = Hyper(**hyper)
    js = JointStep(g, cams, dev(X, torch.float32), dev(obs_point, torch.int32), dev(xy, torch.float32),
                   dev(voff, torch.int64), dev(tg, torch.float32), off, views, h, merged_tracks=merged,
                   dynamic_batch=len(views) > 1, deterministic=deterministic)
    js.ensure_capacity()
    js.capture(warmup=0)     # capturing does not run the step
    for _ in range(replays):
        js.run()
    torch.cuda.synchronize()
    assert js.status_flags() == 0
    return js


@pytest.mark.parametrize("variant", list(VARIANTS) + ["full_deterministic", "merged_tracks_deterministic"])
@pytest.mark.parametrize("kind", ["tiny", "uneven_batch"])
def test_graph_replayed_step_equals_the_oracle_iteration(kind, variant):
    w, views = _workload(kind)
    det = variant.endswith("_deterministic")
    variant = variant.replace("_deterministic", "")
    merged = variant == "merged_tracks"
    hyper = dict(HYPER, **VARIANTS[variant])
    inputs = _inputs(w, merged)
    params, X, wh, K, Rt, targets, obs_point, obs_view, xy, _ = inputs
    js = _gpu_step(w, views, inputs, hyper, merged, deterministic=det)
    V = len(wh)
    exp = oracle.joint_step(params, X, Rt, np.zeros((V, 6)), wh, K, views, targets, obs_point, obs_view, xy, hyper,
                            {}, 1, merged_tracks=merged)
    loss = js.loss.cpu().numpy()
    assert loss[0] == pytest.approx(exp["loss_photo"], rel=1e-4)
    assert loss[1] == pytest.approx(exp["loss_ba"], rel=1e-5, abs=1e-12)
    # the iteration's gradients
    for k, t in zip(KEYS, js.dg.tensors()):
        assert rel_linf(t.cpu().numpy(), exp["grads"][k]) <= 1e-3, k
    if not merged:
        gX = js.gX.cpu().numpy()
        if hyper["lambda_ba"] == 0.0:
            assert not gX.any()
        else:
            assert rel_linf(gX, exp["g_X"]) <= 1e-4
    g_tan = js.g_tan.cpu().numpy()
    for v in views:
        assert pose_rel_err(g_tan[v], exp["tangent"][v], exp["tangent_abs"][v]) <= 1e-3
    # the parameters after the Adam step
    lrs = dict(mean=hyper["lr_mean"], log_scale=hyper["lr_log_scale"], quat=hyper["lr_quat"],
               opacity_logit=hyper["lr_opacity"], sh=hyper["lr_sh"])
    for k, t in zip(KEYS, js.g.tensors()):
        got = t.cpu().numpy().astype(np.float64)
        e = exp["params"][k]
        g = np.abs(exp["grads"][k])
        sure = g >= 1e-2 * g.max()
        np.testing.assert_allclose(got[sure], e[sure], rtol=0, atol=1e-6 * (1.0 + np.abs(e[sure]).max()))
        assert np.abs(got - e).max() <= 2.0 * lrs[k] + 1e-6 * (1.0 + np.abs(e).max()), k
    if not merged:
        np.testing.assert_allclose(js.X.cpu().numpy(), exp["X"], rtol=0, atol=2.0 * hyper["lr_track"] + 1e-6)
    xi = js.xi.cpu().numpy().astype(np.float64)
    if hyper["freeze_poses"]:
        assert not xi.any()
        np.testing.assert_array_equal(js.Rt.cpu().numpy(), Rt.astype(np.float32))
    else:
        # the FP32 Adam step (bias corrections in float) is exact to ~3e-5
        np.testing.assert_allclose(xi, exp["xi"], rtol=1e-4, atol=1e-9)
        np.testing.assert_allclose(js.Rt.cpu().numpy(), exp["Rt"], rtol=0, atol=2e-6)


@pytest.mark.parametrize("merged", [False, True])
def test_deterministic_step_is_bit_identical_across_runs(merged):
    """Two JointSteps from the same state, each replaying its graph three
    times on the uneven batch: with the deterministic backward and track
    term, every parameter, pose and both losses agree bit for bit."""
    w, views = _workload("uneven_batch")
    inputs = _inputs(w, merged)
    outs = []
    for _ in range(2):
        js = _gpu_step(w, views, inputs, HYPER, merged, deterministic=True, replays=3)
        outs.append([t.cpu().numpy().copy() for t in list(js.g.tensors()) + [js.X, js.xi, js.Rt, js.loss,
                                                                             js.g_tan]])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
