"""Parity at the full size of the 8-view 1237x822, 200k-Gaussian SH3
workload, in the batched launch configuration the benchmark times: sampled
pixels and 64 sampled Gaussians against the oracle (which computes them one
by one), the pose tangent and all 200k Gaussians' gradients of a cotangent
on sampled pixels, and the translation gauge identity of all gradients."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import f32, gpu_backward, gpu_forward, knife_mask, oracle_cam, oracle_scene, pose_rel_err, rel_linf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()
    w = synth.make_workload("mid")
    views = list(range(8))
    r, g, cams, batch = gpu_forward(w["scene"], w["wh"], w["K"], w["Rt"], views)
    return w, r, g, cams, batch, oracle_scene(w["scene"])


def test_sampled_pixels_match_oracle(mid):
    w, r, g, cams, batch, osc = mid
    rng = np.random.default_rng(0)
    img = r.image.cpu().numpy()
    for b in (0, 5):
        v = b
        W, H = int(w["wh"][v][0]), int(w["wh"][v][1])
        pix = np.stack([rng.integers(W // 4, 3 * W // 4, 48), rng.integers(H // 4, 3 * H // 4, 48)], 1)
        ref = oracle.render(osc, oracle_cam(w["wh"], w["K"], w["Rt"], v), pixels=pix, knife_eps=1e-4)
        a = int(batch.px_offset_host[b])
        got = img[a + pix[:, 1] * W + pix[:, 0]]
        ok = ~knife_mask(ref)
        assert ok.sum() >= 40
        assert rel_linf(got[ok], ref["image"][ok]) <= 1e-4
        assert (ref["n_added"][ok] > 0).mean() > 0.5


def test_sampled_gaussian_gradients_match_oracle(mid):
    w, r, g, cams, batch, osc = mid
    v = 0
    cam = oracle_cam(w["wh"], w["K"], w["Rt"], v)
    W, H = int(w["wh"][v][0]), int(w["wh"][v][1])
    proj = oracle.project(osc, cam)
    rng = np.random.default_rng(1)
    cand = np.nonzero(proj[:, oracle.P["visible"]] > 0)[0]
    picks = rng.choice(cand, 64, replace=False)
    vimg = np.zeros((batch.n_pixels, 3))
    wv = f32(rng.normal(size=(H, W, 3)))
    rects = []
    for j in picks:
        x0, y0, x1, y1 = (int(proj[j, oracle.P[k]]) for k in ("px_x0", "px_y0", "px_x1", "px_y1"))
        uu, vv = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1))
        pix = np.stack([uu.ravel(), vv.ravel()], 1)
        k = oracle.render(osc, cam, pixels=pix, knife_eps=1e-4)
        bad = knife_mask(k)
        wv[pix[bad, 1], pix[bad, 0]] = 0.0
        rects.append(pix)
    vimg[:W * H] = wv.reshape(-1, 3)
    got = gpu_backward(r, g, v_image=vimg)
    for j, pix in zip(picks, rects):
        e = oracle.render_bwd(osc, cam, wv[pix[:, 1], pix[:, 0]], pixels=pix)
        gj = np.concatenate([got[k][j].ravel() for k in ("mean", "log_scale", "quat", "opacity_logit", "sh")])
        ej = np.concatenate([e[k][j].ravel() for k in ("mean", "log_scale", "quat", "opacity_logit", "sh")])
        assert rel_linf(gj, ej) <= 1e-3, (j, rel_linf(gj, ej))


def sampled_pixel_cotangent(w, r, g, batch, osc, b, n_pix, seed):
    """A random cotangent on n_pix distinct pixels of slot b (knife-edge
    pixels zeroed), zero elsewhere: the GPU's gradients of all Gaussians and
    the view's pose tangent, and the oracle's for exactly those pixels."""
    v = int(batch.views_host[b])
    W, H = int(w["wh"][v][0]), int(w["wh"][v][1])
    rng = np.random.default_rng(seed)
    flat = rng.choice(W * H, n_pix, replace=False)
    pix = np.stack([flat % W, flat // W], 1)
    cam = oracle_cam(w["wh"], w["K"], w["Rt"], v)
    ref = oracle.render(osc, cam, pixels=pix, knife_eps=1e-4)
    vals = f32(rng.normal(size=(n_pix, 3)))
    vals[knife_mask(ref)] = 0.0
    vimg = np.zeros((batch.n_pixels, 3))
    vimg[int(batch.px_offset_host[b]) + flat] = vals
    got = gpu_backward(r, g, v_image=vimg)
    exp = oracle.render_bwd(osc, cam, vals, pixels=pix)
    return got, exp, v


def test_sampled_pixel_cotangent_pose_tangent_and_all_gradients(mid):
    w, r, g, cams, batch, osc = mid
    got, exp, v = sampled_pixel_cotangent(w, r, g, batch, osc, 3, 400, 5)
    for k in ("mean", "log_scale", "quat", "opacity_logit", "sh"):
        assert rel_linf(got[k], exp[k]) <= 1e-3, (k, rel_linf(got[k], exp[k]))
    assert pose_rel_err(got["tangent"][v], exp["tangent"], exp["tangent_abs"]) <= 1e-3
    assert not np.delete(got["tangent"], v, axis=0).any()


def test_translation_gauge_identity_full_size(mid):
    """sum_j dL/dmu_j - sum_i R_i^T dL/drho_i = 0 for any image cotangent
    (the world-translation gauge), on the GPU's own full-size gradients."""
    w, r, g, cams, batch, osc = mid
    rng = np.random.default_rng(2)
    vimg = f32(rng.normal(size=(batch.n_pixels, 3)))
    got = gpu_backward(r, g, v_image=vimg)
    s_mu = got["mean"].sum(0)
    s_t = np.zeros(3)
    for v in range(8):
        R = f32(w["Rt"][v, :9]).reshape(3, 3)
        s_t += R.T @ got["tangent"][v, :3]
    scale = np.abs(got["mean"]).sum(0).max()
    assert np.abs(s_mu - s_t).max() <= 1e-3 * scale
