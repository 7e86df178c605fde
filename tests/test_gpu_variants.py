"""The paper's ablation variants of the joint step: frozen poses,
photometric-only (lambda_BA = 0) and merged tracks (track points are
Gaussian means)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _joint(merged=False, **hyper):
    from paper_2603_04847_gb300 import Cameras, Gaussians, Hyper, JointStep
    w = synth.make_workload("batched", n_gaussians=3000, n_views=5, width=(80, 160), height=(64, 120),
                            n_tracks=200, seed=0)
    wh, K, Rt = w["wh"], w["K"], w["Rt"]
    cams = Cameras.from_numpy(wh, K, Rt)
    g = Gaussians.from_numpy(w["scene"])
    tr = w["tracks"]
    rng = np.random.default_rng(1)
    xy = rng.uniform(10, 60, (len(tr["obs_point"]), 2))
    obs_point = tr["obs_point"]
    if merged:   # track k is Gaussian idx[k]
        idx = rng.choice(g.n, size=int(obs_point.max()) + 1, replace=False)
        obs_point = idx[obs_point].astype(np.int32)
    P = (wh[:, 0] * wh[:, 1]).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(P)])
    targets = torch.as_tensor(np.random.default_rng(2).uniform(0, 1, (int(off[-1]), 3)), dtype=torch.float32,
                              device="cuda")
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    h = dict(lambda_ba=0.1, lr_pose=1e-3, eps=1e-6)
    h.update(hyper)
    js = JointStep(g, cams, dev(tr["X"], torch.float32), dev(obs_point, torch.int32), dev(xy, torch.float32),
                   dev(tr["view_obs_offset"], torch.int64), targets, off, [4, 1, 3], Hyper(**h),
                   merged_tracks=merged)
    js.ensure_capacity()
    return js


def _np(t):
    return t.detach().cpu().numpy().copy()


def test_frozen_poses_keep_the_initial_poses():
    js = _joint(freeze_poses=True)
    T0, mean0 = _np(js.T0), _np(js.g.mean)
    for _ in range(2):
        js.step()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_np(js.Rt), T0)
    assert not np.any(_np(js.xi))
    assert np.abs(_np(js.g.mean) - mean0).max() > 0.0
    assert js.status_flags() == 0


def test_photometric_only_runs_no_track_term():
    js = _joint(lambda_ba=0.0)
    X0 = _np(js.X)
    for _ in range(2):
        js.step()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_np(js.X), X0)
    assert float(js.loss[1].item()) == 0.0 and int(js.n_masked.item()) == 0
    # the Gaussians' first step does not depend on the track term
    a, b = _joint(lambda_ba=0.0), _joint()
    a.step()
    b.step()
    torch.cuda.synchronize()
    for x, y in zip(a.g.tensors(), b.g.tensors()):
        np.testing.assert_allclose(_np(x), _np(y), rtol=1e-4, atol=1e-6)


def test_merged_tracks_add_the_track_gradient_to_the_means():
    """dg.mean of a merged-tracks step = that of the photometric-only step +
    the track term's gradient at the indexed Gaussians' means."""
    from paper_2603_04847_gb300.core import track_reproj_fwd_bwd, track_workspace_bytes
    merged, photo = _joint(merged=True), _joint(lambda_ba=0.0)
    mean0 = merged.g.mean.clone()
    Rt0 = merged.Rt.clone()
    merged.step()
    photo.step()
    torch.cuda.synchronize()
    gX = torch.zeros_like(mean0)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    tan = torch.zeros_like(merged.g_tan)
    nm = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(max(track_workspace_bytes(merged.batch), 256), dtype=torch.uint8, device="cuda")
    h = merged.h
    track_reproj_fwd_bwd(mean0, merged.obs_point, merged.obs_xy, merged.view_obs_offset, merged.cams,
                         merged.batch, h.huber_delta, h.lambda_ba, loss, gX, tan, nm, ws, Rt0)
    torch.cuda.synchronize()
    exp = _np(photo.dg.mean) + _np(gX)
    got = _np(merged.dg.mean)
    assert np.abs(_np(gX)).max() > 0.0
    assert np.abs(got - exp).max() <= 1e-4 * np.abs(exp).max()
    assert abs(float(merged.loss[1].item()) - float(loss.item())) <= 1e-9 * max(1.0, abs(float(loss.item())))
    # the means' Adam group moved the tracked Gaussians (no separate group)
    assert merged.X.data_ptr() == merged.g.mean.data_ptr()
