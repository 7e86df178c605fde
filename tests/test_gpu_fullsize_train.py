"""Parity at the size of the training-loop step: 8 views of 1600x1066 and
3M Gaussians SH3 (the first batch of the 200-view training workload), in
the batched launch configuration the benchmark times: sampled pixels
against the oracle (which computes them one by one), the pose tangent and
all 3M Gaussians' gradients of a cotangent on sampled pixels, and the
translation gauge identity of all gradients."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import f32, gpu_backward, gpu_forward, knife_mask, oracle_cam, oracle_scene, pose_rel_err, rel_linf
from test_gpu_fullsize import sampled_pixel_cotangent

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def train():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()
    w = synth.make_workload("train", n_tracks=100)
    views = list(range(8))
    r, g, cams, batch = gpu_forward(w["scene"], w["wh"], w["K"], w["Rt"], views)
    yield w, r, g, cams, batch, oracle_scene(w["scene"]), views
    del r, g
    torch.cuda.empty_cache()


def test_train_size_sampled_pixels_match_oracle(train):
    w, r, g, cams, batch, osc, views = train
    assert r.n_instances() > 50_000_000   # the size this test is about
    rng = np.random.default_rng(3)
    img = r.image.cpu().numpy()
    for b in (1, 6):
        v = views[b]
        W, H = int(w["wh"][v][0]), int(w["wh"][v][1])
        pix = np.stack([rng.integers(W // 4, 3 * W // 4, 24), rng.integers(H // 4, 3 * H // 4, 24)], 1)
        ref = oracle.render(osc, oracle_cam(w["wh"], w["K"], w["Rt"], v), pixels=pix, knife_eps=1e-4)
        a = int(batch.px_offset_host[b])
        got = img[a + pix[:, 1] * W + pix[:, 0]]
        ok = ~knife_mask(ref)
        assert ok.sum() >= 18
        assert rel_linf(got[ok], ref["image"][ok]) <= 1e-4
        assert (ref["n_added"][ok] > 0).mean() > 0.5


def test_train_size_sampled_pixel_cotangent_pose_tangent_and_all_gradients(train):
    w, r, g, cams, batch, osc, views = train
    got, exp, v = sampled_pixel_cotangent(w, r, g, batch, osc, 5, 64, 6)
    for k in ("mean", "log_scale", "quat", "opacity_logit", "sh"):
        assert rel_linf(got[k], exp[k]) <= 1e-3, (k, rel_linf(got[k], exp[k]))
    assert pose_rel_err(got["tangent"][v], exp["tangent"], exp["tangent_abs"]) <= 1e-3


def test_train_size_translation_gauge_identity(train):
    """sum_j dL/dmu_j - sum_i R_i^T dL/drho_i = 0 for any image cotangent,
    on the GPU's own gradients of all 3M Gaussians and 8 poses."""
    w, r, g, cams, batch, osc, views = train
    rng = np.random.default_rng(4)
    vimg = f32(rng.normal(size=(batch.n_pixels, 3)))
    got = gpu_backward(r, g, v_image=vimg)
    s_mu = got["mean"].sum(0)
    s_t = np.zeros(3)
    for v in views:
        R = f32(w["Rt"][v, :9]).reshape(3, 3)
        s_t += R.T @ got["tangent"][v, :3]
    scale = np.abs(got["mean"]).sum(0).max()
    assert np.abs(s_mu - s_t).max() <= 1e-3 * scale
